"""Kernel-ridge snapshots by multishift CG (subapsnap_krr_snapshots) against the oracle.

The oracle's snapshot matrix (oracle/krr.py::snapshot_matrix) solves every
(K_sigma + lambda I) x = b of the snapshot grid directly in float64.  The device
runs one CG per sigma on the smallest lambda and takes the other lambda values
from the shifted recurrences of the same Krylov space.  Checks:
  * every system reaches the requested true residual (the device's own float64
    residual and the oracle's, recomputed on the host);
  * each column equals the oracle's solution within cond(A) times the residual
    (the forward error bound of a backward-stable residual), with cond from numpy;
  * the grid order: column a * nlambda + b belongs to (sigma_a, lambda_b), the
    order of the workload's snapshot parameters;
  * a ragged N (not a multiple of the 128-row tiles or 64-point chunks), a single
    lambda (plain CG) and a lambda list in decreasing order (the seed is the
    smallest lambda wherever it sits);
  * an iteration limit too small to converge raises SAS_ENOCONV with finite
    iterates.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import krr  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from workloads import get_config  # noqa: E402

TOL = 1e-11


def run(prob, sig, lam, tol=TOL, maxit=5000):
    X = torch.from_numpy(np.ascontiguousarray(prob.X)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(prob.b)).cuda()
    out = torch.full((len(sig) * len(lam), prob.n), float("nan"), dtype=torch.float64, device="cuda")
    its, res = api.subapsnap_krr_snapshots(X, b, sig, lam, out, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    return out.cpu().numpy(), its, res


@pytest.mark.parametrize("N", [400, 333])
def test_snapshot_grid_matches_oracle(N):
    prob = get_config("kernel_ridge", N=N, r=16, s=32, m=4)  # 4 x 4 grid: sigma 0.5..2, lambda 1e-4..1e-1
    sig = np.unique(prob.snap_params[:, 0])
    lam = np.unique(prob.snap_params[:, 1])
    Xd, its, res = run(prob, sig, lam)
    Xo = krr.snapshot_matrix(prob)  # n x r, columns in the order of prob.snap_params
    print(f"N = {N}: iterations {its.tolist()}, device residuals max {res.max():.1e}")
    assert (res <= TOL * 1.01).all()
    for c, p in enumerate(prob.snap_params):
        assert np.isclose(p[0], sig[c // len(lam)]) and np.isclose(p[1], lam[c % len(lam)])
        A = krr.full_matrix(prob.X, p)
        ro = np.linalg.norm(A @ Xd[c] - prob.b) / np.linalg.norm(prob.b)
        assert ro <= 2 * TOL, (c, ro)
        kap = np.linalg.cond(A)
        err = np.linalg.norm(Xd[c] - Xo[:, c]) / np.linalg.norm(Xo[:, c])
        assert err <= 4 * kap * (ro + 1e-15), (c, err, kap, ro)


def test_single_lambda_and_unsorted_grid():
    prob = get_config("kernel_ridge", N=300, r=16, s=32, m=4)
    sig = np.array([1.1, 0.6])
    lam = np.array([1e-1, 3e-3, 1e-2])  # the seed (smallest) sits in the middle
    Xd, its, res = run(prob, sig, lam)
    X1, its1, res1 = run(prob, sig[:1], lam[1:2])  # one system: plain CG
    assert (res <= TOL * 1.01).all() and res1[0] <= TOL * 1.01
    for a, s in enumerate(sig):
        for j, l in enumerate(lam):
            xo = np.linalg.solve(krr.full_matrix(prob.X, (s, l)), prob.b)
            err = np.linalg.norm(Xd[a * len(lam) + j] - xo) / np.linalg.norm(xo)
            assert err <= 1e-8, (s, l, err)
    # the seed system alone takes the same iterations as inside the grid
    assert its1[0] == its[1]
    assert np.linalg.norm(X1[0] - Xd[1]) <= 1e-9 * np.linalg.norm(Xd[1])


def test_iteration_limit_reports_no_convergence():
    prob = get_config("kernel_ridge", N=300, r=16, s=32, m=4)
    X = torch.from_numpy(np.ascontiguousarray(prob.X)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(prob.b)).cuda()
    out = torch.zeros((2, prob.n), dtype=torch.float64, device="cuda")
    with pytest.raises(api.SasError) as ei:
        api.subapsnap_krr_snapshots(X, b, [2.0], [1e-4, 1e-3], out, tol=1e-14, maxit=3)
    assert ei.value.code == api.SAS_ENOCONV
    assert torch.isfinite(out).all().item()
