"""Float64-accurate reconstruction of the mixed form on the tensor cores, against the oracle.

x_hat = S y from 9-bit fixed-point digits of S (one exponent per row, from its
largest entry) and of y (one exponent per parameter, from ||y||_1), fifteen
digit products in the f16 tensor cores and an exact int64 assembly.  Per entry
the distance to the float64 product is bounded by the dropped digit pairs and
the rounding of the tail accumulator; the worst case is below
2^-34 max_k |S_ik| ||y_j||_1 and the typical error ~2^-44 of that scale, below
float64 rounding of S y itself for these shapes.  The oracle's float64 product
(oracle.online.reconstruct) decides.

Shapes: ragged row tiles (n not a multiple of 128) and parameter tiles (m not a
multiple of 128), fewer row tiles than SMs (parameter tiles split into ranges),
long units (many parameter tiles past one resident S tile), r from 1 to 64,
and inputs that drive the digits to their bounds (every sigma_0 at +-512, y with
equal entries, rows and parameters of zeros, scales from 1e-200 to 1e200).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import online  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver  # noqa: E402

from _problems import Case, mixed_bound  # noqa: E402

BOUND = 2.0 ** -34


def reconstruct(case, S, Y, kernel=0):
    """subapsnap_reconstruct on a mixed context whose basis is S (n x r)."""
    p = case.prob
    solver = AffineSolver(p, S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_RECON_KERNEL, kernel)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    out = torch.full((Y.shape[0], p.n), float("nan"), dtype=torch.float64, device="cuda")
    solver.reconstruct(Yd, out)
    st = api.subapsnap_device_status(solver.ctx)
    torch.cuda.synchronize()
    solver.close()
    assert st == 0
    return out.cpu().numpy()


def check_entries(S, Y, X, what=""):
    ref = online.reconstruct(S, Y)
    scale = np.abs(S).max(axis=1)[None, :] * np.abs(Y).sum(axis=1)[:, None]
    err = np.abs(X - ref)
    assert np.isfinite(X).all(), what
    ratio = np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), err)
    worst = float(ratio.max())
    print(f"{what}: max |x - x_oracle| / (max|S_i| ||y||_1) = 2^{np.log2(max(worst, 1e-300)):.1f}")
    assert (err <= BOUND * scale).all(), (what, worst)
    return ref


@pytest.mark.parametrize("N,r,s,m", [(45, 60, 120, 300), (40, 20, 40, 129), (32, 64, 128, 128),
                                     (48, 33, 70, 1), (20, 60, 120, 1000), (12, 1, 4, 777),
                                     (30, 7, 14, 127)])
def test_digit_reconstruction_random(N, r, s, m):
    case = Case("diffusion_2d", basis="random", N=N, r=r, s=s, m=8)
    rng = np.random.default_rng(N * 1000 + r)
    # decaying coefficients, as the coefficients of a snapshot basis decay
    Y = rng.standard_normal((m, r)) * (10.0 ** (-np.arange(r) / 6.0))[None, :]
    X = reconstruct(case, case.S, Y)
    ref = check_entries(case.S, Y, X, f"N={N} r={r} m={m}")
    rel = np.linalg.norm(X - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 2e-12
    # the float64 CUDA-core product of the same context agrees to float64 rounding
    X1 = reconstruct(case, case.S, Y, kernel=1)
    assert (np.abs(X1 - ref) <= 4e-14 * np.abs(case.S).sum(axis=1)[None, :] *
            np.abs(Y).max(axis=1)[:, None]).all()


def test_digit_reconstruction_extreme_inputs():
    """Digits at their bounds and extreme scales: every row of S with all entries
    at +-(1 - 2^-12) of its scale (sigma_0 = +-512 everywhere), rows of zeros,
    row scales from 1e-100 to 1e100; parameters with equal |y_k| (L1 = 64 max),
    a single nonzero coefficient, all zeros, and scales from 1e-100 to 1e100."""
    case = Case("diffusion_2d", basis="random", N=24, r=64, s=128, m=8)
    n, r = case.prob.n, 64
    rng = np.random.default_rng(7)
    signs = rng.choice([-1.0, 1.0], size=(n, r))
    S = signs * (1 - 2.0 ** -12)
    S[1::7] = rng.standard_normal(S[1::7].shape)
    S[3::11] = 0.0
    rowscale = 10.0 ** rng.uniform(-100, 100, size=n)
    S = S * rowscale[:, None]
    m = 300
    Y = rng.standard_normal((m, r))
    Y[0] = 1.0
    Y[1] = -1.0
    Y[2] = 0.0
    Y[3] = 0.0
    Y[3, 17] = 3.5
    Y[4] = np.where(np.arange(r) % 2 == 0, 1.0, -1.0) * (1 + 2.0 ** -9)
    Y[5:40] *= 10.0 ** rng.uniform(-100, 100, size=(35, 1))
    X = reconstruct(case, S, Y)
    ref = check_entries(S, Y, X, "extreme inputs")
    assert (X[2] == 0.0).all() and (X[:, 3::11] == 0.0).all()


def test_mixed_solve_xhat_is_float64_accurate():
    """solve_batch(SAS_OUT_XHAT) in the mixed form: x_hat against the oracle's float64
    answer within the mixed least-squares bound plus 1e-12, and the float32 option
    (SAS_OPT_XHAT_F32) within 2e-6."""
    case = Case("diffusion_2d", N=40, r=60, s=120, m=300)
    p = case.prob
    params = p.test_params
    Yo, rho_o = case.oracle_solve(params)
    Xo = Yo @ case.S.T
    bound = mixed_bound(p, case.S, case.J, params, Yo, rho_o)
    P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    m = params.shape[0]
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    X = torch.full((m, p.n), float("nan"), dtype=torch.float64, device="cuda")
    solver.solve(P, api.SAS_OUT_XHAT, X)
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_XHAT_F32, 1)
    X32 = torch.full((m, p.n), float("nan"), dtype=torch.float32, device="cuda")
    solver.solve(P, api.SAS_OUT_XHAT, X32)
    st = api.subapsnap_device_status(solver.ctx)
    torch.cuda.synchronize()
    solver.close()
    assert st == 0
    e = np.linalg.norm(X.cpu().numpy() - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
    print(f"mixed float64 x_hat vs oracle: max {e.max():.2e} (bound max {bound.max():.2e})")
    assert (e <= bound + 1e-12).all()
    e32 = np.linalg.norm(X32.double().cpu().numpy() - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
    assert e32.max() <= 2e-6


def test_digit_reconstruction_long_units_against_float64_product():
    """n = 262,144 (2048 row tiles: every unit streams all parameter tiles past its
    resident S digits) with m = 2100 (17 parameter tiles, the last ragged): the
    digit kernel against the float64 CUDA-core product on the device, entry by
    entry, and against the oracle on sampled parameters."""
    case = Case("diffusion_2d", basis="random", rows="random", N=512, r=60, s=120, m=8)
    rng = np.random.default_rng(3)
    m = 2100
    Y = rng.standard_normal((m, 60)) * (10.0 ** (-np.arange(60) / 6.0))[None, :]
    p = case.prob
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    Yd = torch.from_numpy(Y).cuda()
    Xtc = torch.full((m, p.n), float("nan"), dtype=torch.float64, device="cuda")
    solver.reconstruct(Yd, Xtc)
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_RECON_KERNEL, 1)
    Xcc = torch.full((m, p.n), float("nan"), dtype=torch.float64, device="cuda")
    solver.reconstruct(Yd, Xcc)
    st = api.subapsnap_device_status(solver.ctx)
    torch.cuda.synchronize()
    solver.close()
    assert st == 0
    Sd = torch.from_numpy(case.S).cuda()
    scale = Sd.abs().amax(dim=1)[None, :] * Yd.abs().sum(dim=1)[:, None]
    err = (Xtc - Xcc).abs()
    assert torch.isfinite(Xtc).all().item()
    assert bool((err <= BOUND * scale + 1e-15 * scale).all().item()), float((err / scale).max())
    pick = [0, 127, 128, 1000, 2047, 2048, 2099]
    check_entries(case.S, Y[pick], Xtc[pick].cpu().numpy(), "long units, sampled parameters")


def test_digit_reconstruction_beyond_float64_range():
    """Entries whose scale 2^{e_i + f_j} puts x outside the normal float64 range take
    the checked path: below it they are flushed to zero (the float64 product is a
    subnormal there), above it they overflow to +-inf as the float64 product does;
    entries of the same launch inside the range stay within the bound."""
    case = Case("diffusion_2d", basis="random", N=16, r=20, s=40, m=8)
    n, r = case.prob.n, 20
    rng = np.random.default_rng(11)
    S = rng.standard_normal((n, r))
    band = np.arange(n) % 3  # 0: normal rows, 1: tiny rows, 2: huge rows
    S[band == 1] *= 1e-250
    S[band == 2] = np.abs(S[band == 2]) * 1e250  # one sign, so that the float64 sum is +inf, not nan
    m = 200
    Y = rng.standard_normal((m, r))
    Y[: m // 2] *= 1e-80   # tiny rows x tiny coefficients underflow
    Y[m // 2:] = np.abs(Y[m // 2:]) * 1e80  # huge rows x huge coefficients overflow
    with np.errstate(over="ignore", invalid="ignore", under="ignore"):
        ref = online.reconstruct(S, Y)
    X = reconstruct(case, S, Y)
    with np.errstate(over="ignore", invalid="ignore", under="ignore"):
        scale = np.abs(S).max(axis=1)[None, :] * np.abs(Y).sum(axis=1)[:, None]
    normal = np.isfinite(scale) & (scale > 1e-290) & (scale < 1e290)
    with np.errstate(invalid="ignore"):  # inf - inf outside the normal entries
        diff = np.abs(X - ref)
    assert (diff[normal] <= BOUND * scale[normal]).all()
    tiny = (scale <= 1e-320)
    assert tiny.any() and (X[tiny] == 0.0).all()
    huge = ~np.isfinite(ref) & ~np.isnan(ref)
    assert huge.any() and (X[huge] == ref[huge]).all()
