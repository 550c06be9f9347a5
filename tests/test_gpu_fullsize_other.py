"""Parity at full size for the transfer-function and kernel-ridge workloads.

The oracle cannot solve every parameter of these batches, so it is compared on
sampled parameters it solves one by one, with the batch solved as bench.py
solves it (one call for the whole batch):
  transfer function, 100^3 grid (n = 10^6, complex), r = 80, s = 200,
    16,384 frequencies, QoI output: y and H(i w) for 10 sampled w, plain
    float64 within 1e-10 (kappa-filtered as elsewhere), mixed within the
    refinement bound;
  delay system, n = 10^7 (Sec. 5.2.3), r = 24, s = 48, 5000 frequencies, QoI
    output: y and H(i w) for 8 sampled w, plain float64 within 1e-10
    (kappa-filtered), mixed within the refinement bound;
  kernel ridge, N = 200,000 points in R^8, r = 100, s = 300, 2048 (sigma,
    lambda): y for 6 sampled parameters, plain float64 within 1e-10; the mixed
    form with tensor-core kernel rows (49 float64 folds per row tile) within
    4 kappa(M) 64 u32 + 1e-10, solved as part of the whole batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import krr, online  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import (AffineSolver, KernelSolver, csr_to_device,  # noqa: E402
                                           select_rows, select_rows_kernel)
from workloads import get_config  # noqa: E402
from workloads import snapshots as wsnap  # noqa: E402

from _problems import mixed_bound  # noqa: E402


def test_transfer_function_full_size():
    prob = get_config("transfer_function")
    blocks = [csr_to_device(A, "cuda") for A in prob.blocks]
    S_rows, res = wsnap.transfer_basis_torch(prob, device="cuda")
    assert res.max() < 1e-8
    J, gaps = select_rows(prob, S_rows, blocks, prob.sel_param, prob.s)
    assert len(set(J.tolist())) == prob.s
    S = S_rows.cpu().numpy().T.copy()
    m = prob.test_params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(prob.test_params)).cuda()
    pick = np.unique(np.concatenate([[0, m // 2, m - 1], np.random.default_rng(2).choice(m, 7, replace=False)]))
    for mode in (api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED):
        solver = AffineSolver(prob, None, J, mode=mode, device="cuda", S_device=S_rows, blocks_device=blocks)
        H = torch.empty(m, dtype=torch.complex128, device="cuda")
        Y = torch.empty((m, prob.r), dtype=torch.complex128, device="cuda")
        flags = torch.zeros(m, dtype=torch.int32, device="cuda")
        solver.solve(P, api.SAS_OUT_QOI, H, flags)
        solver.solve(P, api.SAS_OUT_Y, Y)
        torch.cuda.synchronize()
        H, Y = H.cpu().numpy(), Y.cpu().numpy()
        assert np.isfinite(H).all()
        worst = 0.0
        for j in pick:
            p = prob.test_params[j]
            yo, rho_o = online.solve_one(prob, S, J, p)
            ho = online.qoi(prob, S, yo[None, :])[0]
            M = online.subsampled_matrix(prob, S, J, p)
            sv = np.linalg.svd(M, compute_uv=False)
            kap = sv[0] / sv[-1]
            ey = np.linalg.norm(Y[j] - yo) / np.linalg.norm(yo)
            worst = max(worst, ey)
            if mode == api.SAS_MODE_PLAIN:
                if kap * 1.1e-16 <= 1e-11:
                    assert ey <= 1e-10, (j, ey, kap)
                    assert abs(H[j] - ho) <= 1e-10 * abs(ho) + 1e-12 * np.abs(S.T @ prob.c).max()
            else:
                bound = mixed_bound(prob, S, J, [p], [yo], [rho_o])[0]
                assert ey <= bound, (j, ey, bound)
        print(f"transfer function full size, mode {mode}: max rel err y {worst:.2e}")
        solver.close()


def test_delay_system_full_size():
    prob = get_config("delay_system")
    blocks = [csr_to_device(A, "cuda") for A in prob.blocks]
    S_rows, res = wsnap.delay_basis_torch(prob, device="cuda")
    assert res < 1e-10
    J, gaps = select_rows(prob, S_rows, blocks, prob.sel_param, prob.s)
    assert len(set(J.tolist())) == prob.s
    S = np.ascontiguousarray(S_rows.cpu().numpy().T)
    m = prob.test_params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(prob.test_params)).cuda()
    pick = np.unique(np.concatenate([[0, m // 2, m - 1], np.random.default_rng(5).choice(m, 5, replace=False)]))
    wq = online.qoi_vector(prob, S)
    for mode in (api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED):
        solver = AffineSolver(prob, None, J, mode=mode, device="cuda", S_device=S_rows, blocks_device=blocks)
        H = torch.empty(m, dtype=torch.complex128, device="cuda")
        Y = torch.empty((m, prob.r), dtype=torch.complex128, device="cuda")
        solver.solve(P, api.SAS_OUT_QOI, H)
        solver.solve(P, api.SAS_OUT_Y, Y)
        torch.cuda.synchronize()
        H, Y = H.cpu().numpy(), Y.cpu().numpy()
        assert np.isfinite(H).all()
        worst = 0.0
        for j in pick:
            p = prob.test_params[j]
            yo, rho_o = online.solve_one(prob, S, J, p)
            M = online.subsampled_matrix(prob, S, J, p)
            sv = np.linalg.svd(M, compute_uv=False)
            kap = sv[0] / sv[-1]
            ey = np.linalg.norm(Y[j] - yo) / np.linalg.norm(yo)
            worst = max(worst, ey)
            if mode == api.SAS_MODE_PLAIN:
                if kap * 1.1e-16 <= 1e-11:
                    assert ey <= 1e-10, (j, ey, kap)
                    ho = wq @ yo
                    assert abs(H[j] - ho) <= 1e-10 * abs(ho) + 1e-12 * np.abs(wq).max() * np.abs(yo).max()
            else:
                bound = mixed_bound(prob, S, J, [p], [yo], [rho_o])[0]
                assert ey <= bound, (j, ey, bound)
        print(f"delay system n = 1e7, mode {mode}: max rel err y {worst:.2e}")
        solver.close()


def test_kernel_ridge_full_size():
    prob = get_config("kernel_ridge")
    X = torch.from_numpy(np.ascontiguousarray(prob.X)).cuda()
    S_rows, res = wsnap.kernel_ridge_basis_torch(prob, X, device="cuda", iters=15)
    J, gaps = select_rows_kernel(prob, X, S_rows, prob.sel_param, prob.s)
    assert len(set(J.tolist())) == prob.s
    S = S_rows.cpu().numpy().T.copy()
    m = prob.test_params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(prob.test_params)).cuda()
    solver = KernelSolver(prob, None, J, mode=api.SAS_MODE_PLAIN, device="cuda", S_device=S_rows, X_device=X)
    pick = np.array([0, 1, m // 2, m - 1, 517, 1201])
    Pp = P[torch.from_numpy(pick).cuda()]
    Y = torch.empty((len(pick), prob.r), dtype=torch.float64, device="cuda")
    solver.solve(Pp, api.SAS_OUT_Y, Y)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy()
    for k, j in enumerate(pick):
        yo, _ = krr.solve_one(prob, S, J, prob.test_params[j])
        M = krr.subsampled_matrix(prob.X, S, J, prob.test_params[j])
        sv = np.linalg.svd(M, compute_uv=False)
        kap = sv[0] / sv[-1]
        ey = np.linalg.norm(Y[k] - yo) / np.linalg.norm(yo)
        print(f"kernel ridge full size, parameter {j}: rel err {ey:.2e}, kappa {kap:.2e}")
        if kap * 1.1e-16 <= 1e-11:
            assert ey <= 1e-10
    solver.close()
    # mixed form, tensor-core kernel rows, the whole batch in one call
    mixed = KernelSolver(prob, None, J, mode=api.SAS_MODE_MIXED, device="cuda", S_device=S_rows,
                         X_device=X)
    api.subapsnap_set_option(mixed.ctx, api.SAS_OPT_ASSEMBLY_KERNEL, 2)
    Ym = torch.empty((m, prob.r), dtype=torch.float64, device="cuda")
    mixed.solve(P, api.SAS_OUT_Y, Ym)
    st = api.subapsnap_device_status(mixed.ctx)
    torch.cuda.synchronize()
    assert st == 0
    Ym = Ym.cpu().numpy()
    assert np.isfinite(Ym).all()
    for j in pick:
        yo, _ = krr.solve_one(prob, S, J, prob.test_params[j])
        M = krr.subsampled_matrix(prob.X, S, J, prob.test_params[j])
        sv = np.linalg.svd(M, compute_uv=False)
        kap = sv[0] / sv[-1]
        ey = np.linalg.norm(Ym[j] - yo) / np.linalg.norm(yo)
        print(f"kernel ridge full size, mixed tensor-core rows, parameter {j}: rel err {ey:.2e}")
        assert ey <= 4 * kap * 64 * 2.0 ** -24 + 1e-10
    mixed.close()
