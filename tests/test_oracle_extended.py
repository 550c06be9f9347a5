"""Pin (v): on tiny systems (n <= 64) the oracle's float64 subsampled solve agrees
with a brute-force solve of the same least-squares problem carried out in 50-digit
arithmetic (normal equations, which at 50 digits lose nothing that matters here).

The float64 answer may differ from the exact one by about kappa(M) u, so the test
allows 1e-13 kappa(M) relative error (plus a small floor).
"""
import numpy as np
import pytest

from oracle import online, problem, selection, snapshots  # noqa: E402
from workloads import get_config  # noqa: E402

CASES = [("reaction_diffusion_1d", dict(n=40, r=6, s=12, m=5)),
         ("diffusion_2d", dict(N=7, r=8, s=16, m=5)),
         ("transfer_function", dict(N=3, r=5, s=10, m=5)),
         ("delay_system", dict(n=50, r=5, s=10, m=5))]


def _exact_ls(M, bJ, digits=50):
    # imported here, not at module level: an image without mpmath then skips these
    # tests when they run instead of skipping the module at collection
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(digits):
        Mm = mpmath.matrix([[mpmath.mpc(complex(v)) for v in row] for row in M])
        bm = mpmath.matrix([mpmath.mpc(complex(v)) for v in bJ])
        MH = Mm.H
        y = mpmath.lu_solve(MH * Mm, MH * bm)
        return np.array([complex(y[i]) for i in range(y.rows)])


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_oracle_matches_extended_precision(name, kw):
    prob = get_config(name, **kw)
    assert prob.n <= 64
    S = snapshots.orthonormal_basis(snapshots.snapshot_matrix(prob))
    V = np.asarray(problem.full_matrix(prob, prob.sel_param) @ S)
    J, _ = selection.cpqr_rows(V, prob.s)
    for p in prob.test_params[:3]:
        y, _ = online.solve_one(prob, S, J, p)
        # brute force: the dense A(p), its rows J, times S, all from the definition
        A = np.asarray(problem.full_matrix(prob, p).todense())
        M = A[J, :] @ S
        ye = _exact_ls(M, np.asarray(prob.b)[J])
        kap = np.linalg.cond(M)
        err = np.linalg.norm(y - ye) / np.linalg.norm(ye)
        assert err <= 1e-13 * kap + 1e-14, (err, kap)
