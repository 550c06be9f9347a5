"""Pin: Theorem 4.2's bound on the oracle's subsampled solutions.

For p0, p* with delta >= ||A(p*) - A(p0)||_2 and C = 3 / sigma_min(A(p0) Q_X), if
sigma_min(S U(p0)) > C delta (U(p0) the polar factor of A(p0) Q_X, S the row
subsample), then the subsampled solution's residual is within a factor
1 / (sigma_min(S U(p0)) - C delta) of the best residual over span(Q_X).  The left
side is computed from the oracle's solve; the right side from dense SVDs.
"""
import numpy as np
import pytest

from oracle import online, problem, selection, snapshots
from workloads import get_config


@pytest.mark.parametrize("name,kw", [("reaction_diffusion_1d", dict(n=60, r=6, s=12, m=4)),
                                     ("diffusion_2d", dict(N=8, r=8, s=16, m=4))],
                         ids=["reaction_diffusion_1d", "diffusion_2d"])
def test_theorem_4_2_bound(name, kw):
    prob = get_config(name, **kw)
    Q = snapshots.orthonormal_basis(snapshots.snapshot_matrix(prob))
    p0 = np.atleast_1d(prob.sel_param).astype(float)
    A0 = np.asarray(problem.full_matrix(prob, p0).todense())
    J, _ = selection.cpqr_rows(A0 @ Q, prob.s)
    W, sig, Vh = np.linalg.svd(A0 @ Q, full_matrices=False)
    U0 = W @ Vh  # polar factor of A(p0) Q
    smin_SU = np.linalg.svd(U0[J, :], compute_uv=False).min()
    C = 3.0 / sig.min()
    checked = 0
    rng = np.random.default_rng(5)
    b = np.asarray(prob.b)
    for scale in (1e-5, 1e-4, 1e-3, 1e-2, 3e-2, 1e-1, 3e-1):
        d = rng.standard_normal(p0.shape)
        ps = p0 + scale * d / np.linalg.norm(d)
        As = np.asarray(problem.full_matrix(prob, ps).todense())
        delta = np.linalg.norm(As - A0, 2)
        if not smin_SU > C * delta:
            continue
        y_hat, _ = online.solve_one(prob, Q, J, ps)
        B = As @ Q
        c, *_ = np.linalg.lstsq(B, b, rcond=None)
        best = np.linalg.norm(B @ c - b)
        ratio = np.linalg.norm(B @ y_hat - b) / best
        bound = 1.0 / (smin_SU - C * delta)
        assert ratio <= bound * (1 + 1e-9), (scale, ratio, bound)
        assert ratio >= 1.0 - 1e-9  # the full least squares is optimal over span(Q)
        checked += 1
    assert checked >= 2, "the theorem's condition held for too few perturbations"
