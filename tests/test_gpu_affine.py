"""GPU parity of the affine online stage against the oracle, through the C-ABI.

Tolerances
  plain float64: ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-10 for every parameter
    whose kappa(M) * 1.1e-16 <= 1e-11; two backward-stable float64 solvers
    may differ by ~kappa(M) u, so parameters beyond that bound are checked on
    the residual instead (the count is reported).  Row sets J must match the
    oracle exactly, in order.
  mixed: the float32 factorisation with float64-residual refinement converges
    to the least-squares solution of the perturbed matrix, so its distance to
    the float64 answer is bounded by ~kappa^2 u32 ||r*|| / (||M|| ||y||) plus
    float64 rounding; the test takes 16x that bound plus 1e-11.  The
    subsampled residual must agree with the plain one to 1e-6 relative
    (it is quadratic in the error of y).  x_hat is float64 from the digit
    products on the tensor cores: its distance to the oracle's x_hat is the
    distance of y plus ~1e-13, so the y bound plus 1e-12 applies.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect with -m "not gpu"
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver, basis_to_device, csr_to_device, select_rows  # noqa: E402

from _problems import Case, mixed_bound as _mixed_bound  # noqa: E402

U32 = 2.0 ** -24
DEV = "cuda"


@pytest.fixture(scope="module")
def c0():
    return Case("reaction_diffusion_1d")


@pytest.fixture(scope="module")
def c1_small():
    return Case("diffusion_2d", N=48, r=60, s=120, m=257)


@pytest.fixture(scope="module")
def delay_small():
    return Case("delay_system", n=3000, r=16, s=32, m=120)


@pytest.fixture(scope="module")
def c3_small():
    return Case("transfer_function", N=9, r=20, s=50, m=300)


def run(case, mode, out_kind, params=None, m=None):
    p = case.prob
    params = p.test_params if params is None else params
    m = params.shape[0] if m is None else m
    solver = AffineSolver(p, case.S, case.J, mode=mode, device=DEV)
    P = torch.from_numpy(np.ascontiguousarray(params[:m], dtype=np.float64)).to(DEV)
    cplx = p.complex_valued
    if out_kind == api.SAS_OUT_Y:
        out = torch.empty((m, p.r), dtype=torch.complex128 if cplx else torch.float64, device=DEV)
    elif out_kind == api.SAS_OUT_QOI:
        out = torch.empty(m, dtype=torch.complex128 if cplx else torch.float64, device=DEV)
    else:
        out = torch.empty((m, p.n), dtype=torch.float64, device=DEV)
    flags = torch.zeros(m, dtype=torch.int32, device=DEV)
    rho = torch.empty(m, dtype=torch.float64, device=DEV)
    solver.solve(P, out_kind, out, flags, rho)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), flags.cpu().numpy(), rho.cpu().numpy()
    solver.close()
    return res


def online_solve(prob, S, J, params):
    from oracle import online
    return online.solve_many(prob, S, J, params)


def rel_err_rows(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def plain_parity(case, params=None):
    p = case.prob
    params = p.test_params if params is None else params
    Y, flags, rho = run(case, api.SAS_MODE_PLAIN, api.SAS_OUT_Y, params)
    Yo, rho_o = case.oracle_solve(params)
    err = rel_err_rows(Y, Yo)
    kap = case.kappas(params)
    strict = kap * 1.1e-16 <= 1e-11
    assert strict.sum() > 0
    assert err[strict].max() <= 1e-10, (err[strict].max(), kap[strict].max())
    # beyond the strict range: residual parity
    if (~strict).any():
        np.testing.assert_allclose(rho[~strict], rho_o[~strict], rtol=1e-6, atol=1e-14)
    # rho is relative to ||b_J||: its rounding error is ~kappa(M) u in absolute terms
    assert (np.abs(rho - rho_o) <= 1e-8 * rho_o + 64 * kap * 1.1e-16).all()
    assert not (flags & api.SAS_FLAG_NONFINITE).any()
    return err, kap


def test_c0_row_selection_matches_oracle(c0):
    p = c0.prob
    S_d = basis_to_device(c0.S, DEV)
    blocks = [csr_to_device(A, DEV) for A in p.blocks]
    J, gaps = select_rows(p, S_d, blocks, p.sel_param, p.s)
    np.testing.assert_array_equal(J, c0.J)
    np.testing.assert_allclose(gaps, c0.gaps, rtol=1e-6, atol=1e-12)


def test_c0_plain_parity(c0):
    err, kap = plain_parity(c0)
    print(f"c0 plain: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")


def test_c0_plain_xhat(c0):
    p = c0.prob
    X, flags, rho = run(c0, api.SAS_MODE_PLAIN, api.SAS_OUT_XHAT)
    Yo, _ = c0.oracle_solve(p.test_params)
    Xo = Yo @ c0.S.T
    err = rel_err_rows(X, Xo)
    kap = c0.kappas(p.test_params)
    strict = kap * 1.1e-16 <= 1e-11
    assert err[strict].max() <= 1e-10


def test_c1_small_plain_parity_ragged(c1_small):
    err, kap = plain_parity(c1_small)
    print(f"c1-small plain: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")


def test_c1_small_plain_xhat_and_qoi(c1_small):
    p = c1_small.prob
    X, _, _ = run(c1_small, api.SAS_MODE_PLAIN, api.SAS_OUT_XHAT)
    H, _, _ = run(c1_small, api.SAS_MODE_PLAIN, api.SAS_OUT_QOI)
    Yo, _ = c1_small.oracle_solve(p.test_params)
    Xo = Yo @ c1_small.S.T
    assert rel_err_rows(X, Xo).max() <= 1e-10
    Ho = Xo.mean(axis=1)  # grid mean of x_hat
    np.testing.assert_allclose(H, Ho, rtol=1e-10, atol=1e-14 * np.abs(Ho).max())


def mixed_bound(case, params, Yo, rho_o):
    return _mixed_bound(case.prob, case.S, case.J, params, Yo, rho_o)


@pytest.mark.parametrize("name", ["c0", "c1_small", "c3_small", "delay_small"])
def test_mixed_error_bound_and_equal_residual(name, request):
    case = request.getfixturevalue(name)
    p = case.prob
    params = p.test_params[:200]
    Y, flags, rho = run(case, api.SAS_MODE_MIXED, api.SAS_OUT_Y, params)
    Yo, rho_o = case.oracle_solve(params)
    err = rel_err_rows(Y, Yo)
    bound = mixed_bound(case, params, Yo, rho_o)
    print(f"{name} mixed: max rel err {err.max():.2e}, median {np.median(err):.2e}, "
          f"max err/bound {(err / bound).max():.2e}, stalled {(flags & api.SAS_FLAG_REFINE_STALL).astype(bool).sum()}")
    assert (err <= bound).all()
    kap = case.kappas(params)
    assert (np.abs(rho - rho_o) <= 1e-6 * rho_o + 64 * kap * 1.1e-16).all()
    # REFINE_STALL means refinement failed outright (correction still above 1e-8 |y|)
    assert not (flags & api.SAS_FLAG_REFINE_STALL)[kap < 1e3].any()


def test_c1_small_mixed_xhat(c1_small):
    p = c1_small.prob
    X, _, _ = run(c1_small, api.SAS_MODE_MIXED, api.SAS_OUT_XHAT)
    Yo, rho_o = c1_small.oracle_solve(p.test_params)
    Xo = Yo @ c1_small.S.T
    err = rel_err_rows(X, Xo)
    bound = _mixed_bound(p, c1_small.S, c1_small.J, p.test_params, Yo, rho_o)
    print(f"c1-small mixed x_hat (float64): max rel err {err.max():.2e}, bound max {bound.max():.2e}")
    assert (err <= bound + 1e-12).all()


def test_c3_small_plain_parity_and_qoi(c3_small):
    p = c3_small.prob
    err, kap = plain_parity(c3_small)
    print(f"c3-small plain: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")
    H, _, _ = run(c3_small, api.SAS_MODE_PLAIN, api.SAS_OUT_QOI)
    Yo, _ = c3_small.oracle_solve(p.test_params)
    from oracle import online
    Ho = online.qoi(p, c3_small.S, Yo)
    kap_ok = kap * 1.1e-16 <= 1e-11
    np.testing.assert_allclose(H[kap_ok], Ho[kap_ok], rtol=1e-10, atol=1e-12 * np.abs(Ho).max())


def test_delay_system_plain_parity_qoi_and_selection(delay_small):
    """The delay rule theta = (i omega, -1, -e^{i omega tau}) on (I, A_0, A_1): y, the
    transfer function H = c^T S y and the device row selection against the oracle."""
    case = delay_small
    p = case.prob
    err, kap = plain_parity(case)
    print(f"delay system plain: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")
    H, _, _ = run(case, api.SAS_MODE_PLAIN, api.SAS_OUT_QOI)
    Yo, _ = case.oracle_solve(p.test_params)
    from oracle import online
    Ho = online.qoi(p, case.S, Yo)
    kap_ok = kap * 1.1e-16 <= 1e-11
    np.testing.assert_allclose(H[kap_ok], Ho[kap_ok], rtol=1e-10, atol=1e-12 * np.abs(Ho).max())
    S_d = basis_to_device(case.S, DEV, complex_valued=True)
    blocks = [csr_to_device(A, DEV) for A in p.blocks]
    J, gaps = select_rows(p, S_d, blocks, p.sel_param, p.s)
    near = np.nonzero(case.gaps < 1e-10)[0]
    upto = near[0] if near.size else p.s
    np.testing.assert_array_equal(J[:upto], case.J[:upto])


def test_c3_small_row_selection_complex(c3_small):
    p = c3_small.prob
    S_d = basis_to_device(c3_small.S, DEV, complex_valued=True)
    blocks = [csr_to_device(A, DEV) for A in p.blocks]
    J, gaps = select_rows(p, S_d, blocks, p.sel_param, p.s)
    near = c3_small.gaps < 1e-10
    assert not near.any()
    np.testing.assert_array_equal(J, c3_small.J)


def _three_points(p):
    return p.snap_params[[0, len(p.snap_params) // 2, len(p.snap_params) - 1]]


@pytest.mark.parametrize("which", ["c0", "c1_small", "delay_small"])
def test_union_selection_matches_oracle(which, request):
    """Union of the CPQR picks at three snapshot points (Sec. 4.3.4), real and complex."""
    from oracle import problem as oproblem, selection
    from paper_2510_04825_gb300.solver import select_rows_union
    case = request.getfixturevalue(which)
    p = case.prob
    pts = _three_points(p)
    S_d = basis_to_device(case.S, DEV, complex_valued=p.complex_valued)
    blocks = [csr_to_device(A, DEV) for A in p.blocks]
    Vs = [np.asarray(oproblem.full_matrix(p, pt) @ case.S) for pt in pts]
    assert min(selection.cpqr_rows(V, p.r)[1].min() for V in Vs) > 1e-8  # no near-ties
    U = select_rows_union(p, S_d, blocks, pts, p.r)
    np.testing.assert_array_equal(U, selection.union_rows(Vs, p.r))
    print(f"{which} union of 3 x {p.r} picks: {len(U)} rows")
    # the union is itself a row set: the plain solve on it matches the oracle
    params = p.test_params[:40]
    solver = AffineSolver(p, None, U, mode=api.SAS_MODE_PLAIN, device=DEV, S_device=S_d, blocks_device=blocks)
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    y = torch.empty((len(params), p.r), dtype=torch.complex128 if p.complex_valued else torch.float64, device=DEV)
    solver.solve(P, api.SAS_OUT_Y, y)
    Yo, _ = online_solve(p, case.S, U, params)
    err = rel_err_rows(y.cpu().numpy(), Yo)
    solver.close()
    assert err.max() <= 1e-9, err.max()


def test_nearest_point_solver_matches_oracle(c0):
    """Per-parameter rows from the nearest of three selection points (Sec. 4.3.4)."""
    from oracle import problem as oproblem, selection
    from paper_2510_04825_gb300.solver import NearestPointSolver
    p = c0.prob
    pts = _three_points(p)
    ns = NearestPointSolver(p, c0.S, pts, p.s, mode=api.SAS_MODE_PLAIN, device=DEV)
    Js = [selection.cpqr_rows(np.asarray(oproblem.full_matrix(p, pt) @ c0.S), p.s)[0] for pt in pts]
    for J, Jo in zip(ns.J, Js):
        np.testing.assert_array_equal(J, Jo)
    params = p.test_params
    idx_o = selection.nearest_points(params, pts)
    assert len(set(idx_o.tolist())) == 3
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    y = torch.full((len(params), p.r), float("nan"), dtype=torch.float64, device=DEV)
    rho = torch.empty(len(params), dtype=torch.float64, device=DEV)
    idx = ns.solve(P, api.SAS_OUT_Y, y, None, rho)
    np.testing.assert_array_equal(idx, idx_o)
    Y = y.cpu().numpy()
    for i, J in enumerate(Js):
        g = np.nonzero(idx_o == i)[0]
        Yo, rho_o = online_solve(p, c0.S, J, params[g])
        assert rel_err_rows(Y[g], Yo).max() <= 1e-10
        np.testing.assert_allclose(rho.cpu().numpy()[g], rho_o, rtol=1e-6, atol=1e-14)
    # parameters grouped by point take the slice path: the same answers
    order = np.argsort(idx_o, kind="stable")
    Ps = torch.from_numpy(np.ascontiguousarray(params[order])).to(DEV)
    ys = torch.full_like(y, float("nan"))
    ns.solve(Ps, api.SAS_OUT_Y, ys)
    torch.cuda.synchronize()
    assert torch.equal(ys.cpu(), y.cpu()[torch.from_numpy(order)])
    ns.close()


def test_blocked_householder_path():
    """s x (r+1) too large for shared memory: the row-blocked QR update runs."""
    case = Case("diffusion_2d", basis="random", N=24, r=100, s=300, m=40)
    err, kap = plain_parity(case)
    print(f"blocked path: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")


def test_square_subsample_and_single_parameter():
    case = Case("reaction_diffusion_1d", n=512, r=12, s=12, m=5)
    err, _ = plain_parity(case)
    Y1, _, rho1 = run(case, api.SAS_MODE_PLAIN, api.SAS_OUT_Y, m=1)
    assert Y1.shape == (1, 12)
    assert rho1[0] < 1e-12  # s = r interpolates


def test_true_residual_matches_oracle(c1_small):
    from oracle import online
    p = c1_small.prob
    params = p.test_params[:16]
    Yo, _ = c1_small.oracle_solve(params)
    Xo = np.ascontiguousarray(Yo @ c1_small.S.T)
    solver = AffineSolver(p, c1_small.S, c1_small.J, device=DEV)
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    rho = torch.empty(len(params), dtype=torch.float64, device=DEV)
    solver.true_residual(P, torch.from_numpy(Xo).to(DEV), rho)
    Ysub = torch.from_numpy(np.ascontiguousarray(Yo)).to(DEV)
    rsub = torch.empty(len(params), dtype=torch.float64, device=DEV)
    solver.residual(P, Ysub, rsub)
    torch.cuda.synchronize()
    ref = [online.true_residual(p, prm, x) for prm, x in zip(params, Xo)]
    ref_sub = [online.subsampled_residual(p, c1_small.S, c1_small.J, prm, y) for prm, y in zip(params, Yo)]
    np.testing.assert_allclose(rho.cpu().numpy(), ref, rtol=1e-6)
    np.testing.assert_allclose(rsub.cpu().numpy(), ref_sub, rtol=1e-6, atol=1e-15)
    solver.close()


def test_invalid_arguments_raise():
    case = Case("reaction_diffusion_1d", n=256, r=8, s=16, m=4)
    p = case.prob
    J = case.J.copy()
    J[3] = J[2]
    with pytest.raises(api.SasError) as ei:
        AffineSolver(p, case.S, J, device=DEV)
    assert ei.value.code == api.SAS_EINVAL
    J = case.J.copy()
    J[0] = p.n
    with pytest.raises(api.SasError):
        AffineSolver(p, case.S, J, device=DEV)
    solver = AffineSolver(p, case.S, case.J, device=DEV)
    P = torch.zeros((0, 1), dtype=torch.float64, device=DEV)
    out = torch.zeros((1, p.r), dtype=torch.float64, device=DEV)
    api.subapsnap_solve_batch(solver.ctx, P, 0, api.SAS_OUT_Y, out)  # m = 0: no-op
    with pytest.raises(api.SasError):
        api.subapsnap_solve_batch(solver.ctx, P, 1, 7, out)
    solver.close()


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED])
def test_every_ls_variant_and_autotune(c1_small, mode):
    """Every launch shape the autotuner may pick gives the oracle's answer."""
    case = c1_small
    p = case.prob
    params = p.test_params[:100]
    Yo, rho_o = case.oracle_solve(params)
    # plain: 5 shared-memory shapes + 1 register-resident; mixed: 5 shapes with float64 M
    # in shared memory, 5 without, 2 register-resident, 5 with M in a global slot per CTA,
    # 9 blocked (panels of 8 reflectors applied to register-resident trailing columns;
    # the panel factorised by the CTA, by warp 0 alone, or by warp 0 with the panel and
    # the refinement corrections in registers)
    nvar = 6 if mode == api.SAS_MODE_PLAIN else 26
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    solver = AffineSolver(p, case.S, case.J, mode=mode, device=DEV)
    bound = _mixed_bound(p, case.S, case.J, params, Yo, rho_o)
    for v in range(nvar):
        api.subapsnap_set_option(solver.ctx, api.SAS_OPT_LS_VARIANT, v)
        Y = torch.empty((len(params), p.r), dtype=torch.float64, device=DEV)
        solver.solve(P, api.SAS_OUT_Y, Y)
        torch.cuda.synchronize()
        err = rel_err_rows(Y.cpu().numpy(), Yo)
        if mode == api.SAS_MODE_PLAIN:
            assert err.max() <= 1e-10, (v, err.max())
        else:
            assert (err <= bound).all(), (v, err.max())
    chosen, times = api.subapsnap_autotune(solver.ctx, P, len(params), 2)
    print(f"autotune mode {mode}: chosen {chosen}, times {[round(t, 4) for t in times[:nvar]]}")
    assert 0 <= chosen < nvar and times[chosen] > 0
    solver.close()


def test_blocked_variants_reject_what_does_not_fit():
    """A blocked variant whose registers cannot hold a trailing column (s > G E) and
    every blocked variant on a complex context are refused, not run."""
    case = Case("diffusion_2d", basis="random", rows="random", N=30, r=20, s=300, m=4)
    P = torch.from_numpy(np.ascontiguousarray(case.prob.test_params)).to(DEV)
    solver = AffineSolver(case.prob, case.S, case.J, mode=api.SAS_MODE_MIXED, device=DEV)
    for v in range(17, 26):  # s = 300 > 256 >= G E for every blocked shape
        api.subapsnap_set_option(solver.ctx, api.SAS_OPT_LS_VARIANT, v)
        Y = torch.empty((4, 20), dtype=torch.float64, device=DEV)
        with pytest.raises(api.SasError):
            solver.solve(P, api.SAS_OUT_Y, Y)
    solver.close()


def test_global_slot_variants_complex(c3_small):
    """Mixed complex solve with the float64 M kept in a global slot per CTA."""
    case = c3_small
    p = case.prob
    params = p.test_params[:60]
    Yo, rho_o = case.oracle_solve(params)
    bound = _mixed_bound(p, case.S, case.J, params, Yo, rho_o)
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device=DEV)
    for v in range(12, 17):
        api.subapsnap_set_option(solver.ctx, api.SAS_OPT_LS_VARIANT, v)
        Y = torch.empty((len(params), p.r), dtype=torch.complex128, device=DEV)
        solver.solve(P, api.SAS_OUT_Y, Y)
        torch.cuda.synchronize()
        err = rel_err_rows(Y.cpu().numpy(), Yo)
        assert (err <= bound).all(), (v, err.max())
    solver.close()


def test_bounded_wait_times_out_and_context_survives():
    """A wait on a barrier nothing arrives on gives up, records SAS_ETIMEOUT and returns;
    the context then solves as before (no GPU fault, no hang)."""
    case = Case("reaction_diffusion_1d", n=256, r=8, s=16, m=4)
    solver = AffineSolver(case.prob, case.S, case.J, device=DEV)
    assert api.subapsnap_selftest_wait(solver.ctx, 0.2) == api.SAS_ETIMEOUT
    assert api.subapsnap_device_status(solver.ctx) == api.SAS_OK  # the word was cleared
    err, _ = plain_parity(case)
    assert err.max() <= 1e-10
    solver.close()


def test_blocked_householder_path_complex():
    """Complex s x (r+1) = 200 x 81 does not fit shared memory: row-blocked QR update."""
    case = Case("transfer_function", basis="random", N=9, r=80, s=200, m=40)
    err, kap = plain_parity(case)
    print(f"blocked complex path: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED])
def test_register_variants_on_c0_and_multichunk(c0, mode):
    """The register-resident and blocked shapes on the 1-D workload (s = 40, r = 20):
    ragged row ownership (40 rows over 4 or 8 lanes), unused column slots, a last
    panel of 4 columns."""
    p = c0.prob
    params = p.test_params[:300]
    Yo, rho_o = c0.oracle_solve(params)
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    solver = AffineSolver(p, c0.S, c0.J, mode=mode, device=DEV)
    variants = [5] if mode == api.SAS_MODE_PLAIN else [10, 11] + list(range(17, 26))
    bound = _mixed_bound(p, c0.S, c0.J, params, Yo, rho_o)
    kap = c0.kappas(params)
    for v in variants:
        api.subapsnap_set_option(solver.ctx, api.SAS_OPT_LS_VARIANT, v)
        Y = torch.empty((len(params), p.r), dtype=torch.float64, device=DEV)
        rho = torch.empty(len(params), dtype=torch.float64, device=DEV)
        solver.solve(P, api.SAS_OUT_Y, Y, None, rho)
        torch.cuda.synchronize()
        err = rel_err_rows(Y.cpu().numpy(), Yo)
        if mode == api.SAS_MODE_PLAIN:
            assert err.max() <= 1e-10, (v, err.max())
        else:
            assert (err <= bound).all(), (v, err.max())
        assert (np.abs(rho.cpu().numpy() - rho_o) <= 1e-6 * rho_o + 64 * kap * 1.1e-16).all()
    solver.close()


@pytest.mark.parametrize("N,r,s", [(24, 29, 97), (30, 60, 128)], ids=["s97_r29", "s128_r60"])
def test_register_panel_variant_edges(N, r, s):
    """The register-panel variant (each lane holding four rows of the panel and of the
    correction vector) at its edges: s = 97 leaves one valid row in the last owning lane
    and r = 29 a last panel of 5 columns; s = 128 fills all 32 lanes."""
    case = Case("diffusion_2d", basis="random", N=N, r=r, s=s, m=40)
    p = case.prob
    params = p.test_params
    Yo, rho_o = case.oracle_solve(params)
    P = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device=DEV)
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_LS_VARIANT, 25)
    Y = torch.empty((len(params), p.r), dtype=torch.float64, device=DEV)
    rho = torch.empty(len(params), dtype=torch.float64, device=DEV)
    solver.solve(P, api.SAS_OUT_Y, Y, None, rho)
    torch.cuda.synchronize()
    err = rel_err_rows(Y.cpu().numpy(), Yo)
    bound = _mixed_bound(p, case.S, case.J, params, Yo, rho_o)
    kap = case.kappas(params)
    print(f"register panel s={s} r={r}: max rel err {err.max():.2e}, kappa max {kap.max():.2e}")
    assert (err <= bound).all(), err.max()
    assert (np.abs(rho.cpu().numpy() - rho_o) <= 1e-6 * rho_o + 64 * kap * 1.1e-16).all()
    solver.close()
