"""Parity at the learned-surrogate workload's full size: 2-D diffusion on the 4096 x 4096
grid (n = 16,777,216), r = 60, s = 120, the 65,536 test parameters, QoI = grid mean and
x_hat for 256 of them (the launch configuration bench.py --workload surrogate times).

The oracle cannot solve 65,536 parameters or store 256 n-vectors, so it is compared on
sampled outputs it computes one by one (oracle.online on the host copy of S):
  * y for 8 parameters spread over the batch: 1e-10 relative, or 16 kappa(M) (dM/||M|| + u)
    where the two float64 assemblies of M (the oracle's explicit rows, the device's affine
    blocks, whose rows cancel terms of size h^-2 |S| with h^-2 = 1.7e7 here) differ by dM
    enough to move two backward-stable solves apart; mixed: also the refinement bound of
    tests/_problems.mixed_bound;
  * the grid-mean QoI (1/n) 1^T x_hat of those parameters, against the oracle's
    qoi(S, y) (relative to |H|, the same tolerances);
  * x_hat at 4096 sampled rows of three parameters of the 256 (float64 in both forms,
    relative to ||x||_inf, the same tolerances);
  * the surrogate's gate: a briefly trained network's predictions for 48 parameters are
    scored by the oracle's float64 subsampled residual ||M y_hat - b_J|| / ||b_J||, and
    the device's accept / fall-back decisions (SAS_FLAG_SURROGATE / SAS_FLAG_FALLBACK)
    must agree with "residual <= tolerance" wherever the oracle's residual is farther from
    the tolerance than two float64 assemblies of M (explicit rows, affine blocks) can
    differ, at the workload's 1e-6 and at the median residual (so that both decisions
    occur); accepted parameters return the prediction, the others the least-squares y.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import online  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver, csr_to_device, select_rows  # noqa: E402
from workloads import get_config  # noqa: E402
from workloads import snapshots as wsnap  # noqa: E402

from _problems import mixed_bound  # noqa: E402

NX = 256


@pytest.fixture(scope="module")
def big():
    prob = get_config("surrogate_diffusion_2d")  # N = 4096, r = 60, s = 120, m = 65536
    blocks = [csr_to_device(A, "cuda") for A in prob.blocks]
    S_rows, res = wsnap.diffusion_basis_torch(prob, device="cuda")
    assert res.max() < 1e-9
    J, _ = select_rows(prob, S_rows, blocks, prob.sel_param, prob.s)
    S = np.ascontiguousarray(S_rows.cpu().numpy().T)  # n x r on the host for the oracle
    return prob, blocks, S_rows, S, J


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED], ids=["plain", "mixed"])
def test_surrogate_workload_full_size_sampled(big, mode):
    prob, blocks, S_rows, S, J = big
    solver = AffineSolver(prob, None, J, mode=mode, device="cuda", S_device=S_rows, blocks_device=blocks)
    m, n = prob.test_params.shape[0], prob.n
    P = torch.from_numpy(np.ascontiguousarray(prob.test_params)).cuda()
    H = torch.empty(m, dtype=torch.float64, device="cuda")
    flags = torch.zeros(m, dtype=torch.int32, device="cuda")
    solver.solve(P, api.SAS_OUT_QOI, H, flags)
    Y = torch.empty((m, prob.r), dtype=torch.float64, device="cuda")
    solver.solve(P, api.SAS_OUT_Y, Y)
    X = torch.empty((NX, n), dtype=torch.float64, device="cuda")
    solver.solve(P[:NX].contiguous(), api.SAS_OUT_XHAT, X)
    st = api.subapsnap_device_status(solver.ctx)
    torch.cuda.synchronize()
    assert st == 0
    assert torch.isfinite(H).all().item() and torch.isfinite(X).all().item()
    fl = flags.cpu().numpy()
    assert not (fl & (api.SAS_FLAG_ILLCOND | api.SAS_FLAG_NONFINITE)).any()
    rng = np.random.default_rng(9)
    pick = np.unique(np.concatenate([[0, 1, NX - 1, m - 1], rng.choice(m, 4, replace=False)]))
    rows = np.sort(rng.choice(n, 4096, replace=False))
    rows_t = torch.from_numpy(rows).cuda()
    Yh, Hh = Y.cpu().numpy(), H.cpu().numpy()
    wq = online.qoi_vector(prob, S)
    for j in pick:
        yo, rho_o = online.solve_one(prob, S, J, prob.test_params[j])
        ey = np.linalg.norm(Yh[j] - yo) / np.linalg.norm(yo)
        ho = float(yo @ wq)
        eh = abs(Hh[j] - ho) / abs(ho)
        # two float64 least-squares solvers on matrices assembled two ways (explicit rows of
        # A(p) against sum_k theta_k (A_k)_J S, whose rows cancel terms of size h^-2 |S|)
        # differ by ~kappa(M) dM / ||M||: the 1e-10 bound holds where that is small, and
        # 16 kappa (dM / ||M|| + u) bounds the rest
        th = np.concatenate([[1.0], prob.test_params[j]])
        M_rows = online.subsampled_matrix(prob, S, J, prob.test_params[j])
        M_aff = sum(t * np.asarray(A[J] @ S) for t, A in zip(th, prob.blocks))
        sv = np.linalg.svd(M_rows, compute_uv=False)
        kap = sv[0] / sv[-1]
        dM = np.linalg.norm(M_rows - M_aff, 2) / sv[0]
        tol = max(1e-10, 16 * kap * (dM + 1.1e-16))
        if mode == api.SAS_MODE_MIXED:
            tol = max(tol, mixed_bound(prob, S, J, prob.test_params[j:j + 1], [yo], [rho_o])[0])
        print(f"4096^2 mode {mode} parameter {j}: y rel err {ey:.2e}, QoI rel err {eh:.2e} "
              f"(kappa {kap:.1e}, assembly dM/||M|| {dM:.1e}, tol {tol:.1e})")
        assert ey <= tol and eh <= tol
        if j < NX and j in (0, 1, NX - 1):
            xs = X[j].index_select(0, rows_t).cpu().numpy()
            xo = S[rows] @ yo
            ex = np.abs(xs - xo).max() / np.abs(xo).max()
            print(f"   x_hat sampled rows rel err {ex:.2e}")
            assert ex <= tol
    solver.close()


def test_surrogate_gate_decisions_match_oracle_residual(big):
    prob, blocks, S_rows, S, J = big
    solver = AffineSolver(prob, None, J, mode=api.SAS_MODE_MIXED, device="cuda", S_device=S_rows,
                          blocks_device=blocks)
    ntrain = 20000
    Ptr = torch.from_numpy(np.random.default_rng(123).uniform(0.0, 1.0, (ntrain, prob.dp))).cuda()
    Ytr = torch.empty((ntrain, prob.r), dtype=torch.float64, device="cuda")
    solver.solve(Ptr, api.SAS_OUT_Y, Ytr)
    api.subapsnap_surrogate_train(solver.ctx, Ptr, Ytr, 8, 1024, 1e-3, seed=7)
    params = np.ascontiguousarray(prob.test_params[:48])
    P = torch.from_numpy(params).cuda()
    Yhat = torch.empty((48, prob.r), dtype=torch.float64, device="cuda")
    api.subapsnap_surrogate_predict(solver.ctx, P, 48, Yhat)
    torch.cuda.synchronize()
    yhat = Yhat.cpu().numpy()
    rho_o = np.array([online.subsampled_residual(prob, S, J, p, y) for p, y in zip(params, yhat)])
    # the residual is sensitive to the rounding of the assembly (each row of A_J S cancels
    # terms of size h^-2 |S|): a decision counts only where the oracle's residual is farther
    # from the tolerance than the discrepancy of two float64 assemblies (explicit rows
    # against sum_k theta_k (A_k)_J S) can move it
    bJn = np.linalg.norm(prob.b[J])
    band = []
    for p, y in zip(params, yhat):
        th = np.concatenate([[1.0], p])
        M_rows = online.subsampled_matrix(prob, S, J, p)
        M_aff = sum(t * np.asarray(A[J] @ S) for t, A in zip(th, prob.blocks))
        dM = np.linalg.norm(M_rows - M_aff, 2) + 1.1e-16 * np.linalg.norm(M_rows, 2)
        band.append(8 * dM * np.linalg.norm(y) / bJn)
    band = np.array(band)
    for tol in (1e-6, float(np.median(rho_o))):
        Y = torch.empty((48, prob.r), dtype=torch.float64, device="cuda")
        flags = torch.zeros(48, dtype=torch.int32, device="cuda")
        rho = torch.empty(48, dtype=torch.float64, device="cuda")
        acc = api.subapsnap_solve_batch_surrogate(solver.ctx, P, 48, api.SAS_OUT_Y, Y, flags, rho, tol)
        torch.cuda.synchronize()
        fl, Yd = flags.cpu().numpy(), Y.cpu().numpy()
        accepted = (fl & api.SAS_FLAG_SURROGATE) != 0
        fell_back = (fl & api.SAS_FLAG_FALLBACK) != 0
        assert (accepted ^ fell_back).all() and accepted.sum() == acc
        clear = np.abs(rho_o - tol) > 1e-6 * tol + band
        assert clear.sum() >= 24
        np.testing.assert_array_equal(accepted[clear], (rho_o <= tol)[clear])
        assert np.array_equal(Yd[accepted], yhat[accepted])
        for j in np.nonzero(fell_back)[0][:3]:
            yo, _ = online.solve_one(prob, S, J, params[j])
            assert np.linalg.norm(Yd[j] - yo) / np.linalg.norm(yo) <= 1e-8
        print(f"gate {tol:.2e}: accepted {acc} of 48; oracle residuals {rho_o.min():.2e} .. {rho_o.max():.2e}")
    solver.close()
