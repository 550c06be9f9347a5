"""GPU parity of the Gaussian-kernel (kernel ridge regression) family.

M(sigma, lambda) = K_sigma(X_J, X) S + lambda S_J is formed on the device
from the points, for every parameter (Sec. 5.3), then solved as the affine
family is.  Tolerances:
  plain float64: y within 1e-10 relative of the oracle for every parameter
    with kappa(M) 1.1e-16 <= 1e-11 (the float64 parity rule of the other tests).
  mixed: the kernel entries are formed in float32 (hi/lo coordinate
    differences, ex2.approx), then either summed on the CUDA cores (float32
    per chunk, chunks added in float64) or on the tensor cores (entries and S
    split into tf32 hi/lo, three products, float32 TMEM sums folded into
    float64 every 4096 points); both leave M with a relative error
    eps_M <= 64 u32.  The solve is refined against that M, so
    ||y - y_oracle|| / ||y|| <= 4 kappa(M) eps_M + the refinement bound.
    The subsampled residual of the plain path (float64 kernel rows) is
    checked against the oracle as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import krr, selection, snapshots as osnap  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import KernelSolver  # noqa: E402
from workloads import get_config  # noqa: E402
from workloads import snapshots as wsnap  # noqa: E402

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def krr_case():
    prob = get_config("kernel_ridge", N=2500, r=16, s=48, m=70)
    S = wsnap.basis(prob)
    V = krr.full_matrix(prob.X, prob.sel_param) @ S
    J, gaps = selection.cpqr_rows(V, prob.s)
    return prob, S, J


def run(prob, S, J, mode, out_kind, params, assembly=0):
    solver = KernelSolver(prob, S, J, mode=mode, device="cuda")
    if mode == api.SAS_MODE_MIXED:
        api.subapsnap_set_option(solver.ctx, api.SAS_OPT_ASSEMBLY_KERNEL, assembly)
    m = params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    if out_kind == api.SAS_OUT_Y:
        out = torch.empty((m, prob.r), dtype=torch.float64, device="cuda")
    else:
        out = torch.empty((m, prob.n), dtype=torch.float64, device="cuda")
    flags = torch.zeros(m, dtype=torch.int32, device="cuda")
    rho = torch.empty(m, dtype=torch.float64, device="cuda")
    solver.solve(P, out_kind, out, flags, rho)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), flags.cpu().numpy(), rho.cpu().numpy(), solver
    return res


def test_kernel_rows_plain_parity(krr_case):
    prob, S, J = krr_case
    params = prob.test_params
    Y, flags, rho, solver = run(prob, S, J, api.SAS_MODE_PLAIN, api.SAS_OUT_Y, params)
    Yo, rho_o = krr.solve_many(prob, S, J, params)
    err = np.linalg.norm(Y - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
    kap = np.array([np.linalg.cond(krr.subsampled_matrix(prob.X, S, J, p)) for p in params])
    strict = kap * 1.1e-16 <= 1e-11
    print(f"kernel plain: max rel err {err[strict].max():.2e}, kappa max {kap.max():.2e}, "
          f"{(~strict).sum()} beyond the strict range")
    assert strict.sum() > 0
    assert err[strict].max() <= 1e-10
    assert (np.abs(rho - rho_o) <= 1e-8 * rho_o + 64 * kap * 1.1e-16).all()
    # standalone residual entry point on the oracle's y
    rr = torch.empty(len(params), dtype=torch.float64, device="cuda")
    solver.residual(torch.from_numpy(np.ascontiguousarray(params)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(Yo)).cuda(), rr)
    torch.cuda.synchronize()
    assert (np.abs(rr.cpu().numpy() - rho_o) <= 1e-8 * rho_o + 64 * kap * 1.1e-16).all()
    solver.close()


@pytest.mark.parametrize("kernel", [1, 2])
def test_kernel_rows_mixed_error(krr_case, kernel):
    prob, S, J = krr_case
    params = prob.test_params
    Y, flags, rho, solver = run(prob, S, J, api.SAS_MODE_MIXED, api.SAS_OUT_Y, params, kernel)
    Yo, rho_o = krr.solve_many(prob, S, J, params)
    err = np.linalg.norm(Y - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
    kap = np.array([np.linalg.cond(krr.subsampled_matrix(prob.X, S, J, p)) for p in params])
    bound = 4 * kap * 64 * U32 + 1e-10
    print(f"kernel mixed ({'tensor' if kernel == 2 else 'CUDA'} cores): max rel err {err.max():.2e}, "
          f"median {np.median(err):.2e}, "
          f"max err/bound {(err / bound).max():.2e}")
    assert (err <= bound).all()
    solver.close()


def test_kernel_rows_xhat(krr_case):
    prob, S, J = krr_case
    params = prob.test_params[:9]
    X, _, _, solver = run(prob, S, J, api.SAS_MODE_PLAIN, api.SAS_OUT_XHAT, params)
    Yo, _ = krr.solve_many(prob, S, J, params)
    Xo = Yo @ S.T
    assert (np.linalg.norm(X - Xo, axis=1) / np.linalg.norm(Xo, axis=1)).max() <= 1e-10
    solver.close()


@pytest.mark.parametrize("N,d,r,s,m", [(9001, 8, 36, 150, 37), (5000, 5, 25, 130, 8),
                                       (3000, 13, 16, 40, 3), (700, 2, 16, 20, 1)])
def test_tensor_core_rows_shapes(N, d, r, s, m):
    """Tensor-core kernel rows on ragged shapes: N not a multiple of the 32-point
    chunk, several 4096-point float64 folds (N = 9001), J tiles with a ragged
    last tile (s = 150, 130), coordinate dimensions padded to multiples of 4
    (d = 5, 13, 2), an odd number of parameters (the last pair has one live
    member) and a single parameter.  Random orthonormal S and random rows J
    (the online stage accepts any); both assembly kernels against the oracle."""
    prob = get_config("kernel_ridge", N=N, d=d, r=r, s=s, m=m)
    rng = np.random.default_rng(N)
    S = wsnap.orthonormalise(rng.standard_normal((N, r)))
    J = np.sort(rng.choice(N, s, replace=False))
    params = prob.test_params
    Yo, _ = krr.solve_many(prob, S, J, params)
    kap = np.array([np.linalg.cond(krr.subsampled_matrix(prob.X, S, J, p)) for p in params])
    bound = 4 * kap * 64 * U32 + 1e-10
    errs = {}
    for kernel in (1, 2):
        Y, flags, rho, solver = run(prob, S, J, api.SAS_MODE_MIXED, api.SAS_OUT_Y, params, kernel)
        st = api.subapsnap_device_status(solver.ctx)
        solver.close()
        assert st == 0
        assert np.isfinite(Y).all()
        errs[kernel] = np.linalg.norm(Y - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
        assert (errs[kernel] <= bound).all(), (kernel, errs[kernel].max(), bound.min())
    print(f"N={N} d={d} s={s} m={m}: max rel err CUDA cores {errs[1].max():.2e}, "
          f"tensor cores {errs[2].max():.2e}, kappa max {kap.max():.2e}")
