"""Leverage-score row selection with weights on the device (Sec. 4.3.2-4.3.3).

  * scores of [A(p_sel) S, b] by shifted CholeskyQR3 on the device against the
    oracle's thin-QR scores, real and complex families (cases where b is not
    numerically in span(A(p_sel) S), so that the scores are well-posed), and on an
    [A(p_sel) S, b] that is numerically rank-deficient: scores that still sum to
    r + 1, without a failure;
  * the weighted online solve (rows of M and b_J scaled by the sampling weights)
    against the oracle's weighted least squares: plain float64 within 1e-10
    (kappa-filtered), the weighted subsampled residual within 1e-8, the mixed form
    within its refinement bound;
  * the residual band (1 -/+ eps) of the weighted subsampled residual contains the
    true residual at the sampling parameter in most draws.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import leverage, online, problem  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import (AffineSolver, basis_to_device, csr_to_device,  # noqa: E402
                                           leverage_rows)

from _problems import Case, U32  # noqa: E402

CASES = [("diffusion_2d", dict(N=20, r=8, s=40, m=30)),
         ("delay_system", dict(n=2000, r=8, s=40, m=30)),
         ("transfer_function", dict(N=6, r=6, s=30, m=20))]


def device_inputs(case):
    p = case.prob
    cplx = bool(p.complex_valued)
    return basis_to_device(case.S, "cuda", cplx), [csr_to_device(A, "cuda") for A in p.blocks]


@pytest.mark.parametrize("name,kw", CASES)
def test_device_scores_match_oracle(name, kw):
    case = Case(name, rows="random", **kw)
    p = case.prob
    V = np.column_stack([np.asarray(problem.full_matrix(p, p.sel_param) @ case.S), p.b])
    sv = np.linalg.svd(V, compute_uv=False)
    assert sv[-1] > 1e-8 * sv[0]  # well-posed scores: b not numerically in span(A(p_sel) S)
    lev_o = leverage.leverage_scores(V)
    S_d, blocks = device_inputs(case)
    u = np.random.default_rng(1).uniform(size=p.s)
    J, w, scores = leverage_rows(p, S_d, blocks, p.sel_param, p.s, u)
    np.testing.assert_allclose(scores, lev_o, rtol=1e-8, atol=1e-12 * lev_o.max())
    assert abs(scores.sum() - (p.r + 1)) < 1e-8 * (p.r + 1)
    Jo, wo = leverage.sample_rows(scores, p.s, u)  # same scores, same uniforms
    np.testing.assert_array_equal(J, Jo)
    np.testing.assert_array_equal(w, wo)


def weighted_bound(p, S, J, w, params, Yo, rho_o):
    """The mixed refinement bound of the weighted system W M(p)."""
    out = []
    bJw = p.b[J] * w
    for prm, y, rr in zip(params, Yo, rho_o):
        M = online.subsampled_matrix(p, S, J, prm) * w[:, None]
        sv = np.linalg.svd(M, compute_uv=False)
        kap = sv[0] / sv[-1]
        rstar = rr * np.linalg.norm(bJw)
        out.append(1e-11 + 16 * (kap ** 2 * U32 * rstar / (sv[0] * np.linalg.norm(y)) + kap * 1.1e-16))
    return np.array(out), None


@pytest.mark.parametrize("name,kw", CASES)
def test_weighted_solve_parity(name, kw):
    case = Case(name, rows="random", **kw)
    p = case.prob
    S_d, blocks = device_inputs(case)
    u = np.random.default_rng(2).uniform(size=p.s)
    J, w, _ = leverage_rows(p, S_d, blocks, p.sel_param, p.s, u)
    params = p.test_params
    Yo, rho_o = online.solve_many(p, case.S, J, params, w=w)
    ydt = torch.complex128 if p.complex_valued else torch.float64
    P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    for mode in (api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED):
        sv = AffineSolver(p, None, J, mode=mode, S_device=S_d, blocks_device=blocks, weights=w)
        Y = torch.empty((len(params), p.r), dtype=ydt, device="cuda")
        rho = torch.empty(len(params), dtype=torch.float64, device="cuda")
        sv.solve(P, api.SAS_OUT_Y, Y, None, rho)
        torch.cuda.synchronize()
        Y, rho = Y.cpu().numpy(), rho.cpu().numpy()
        sv.close()
        err = np.linalg.norm(Y - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
        if mode == api.SAS_MODE_PLAIN:
            kap = np.array([np.linalg.cond(online.subsampled_matrix(p, case.S, J, q) * w[:, None])
                            for q in params])
            ok = kap * 1.1e-16 <= 1e-11
            assert ok.sum() > 0
            assert err[ok].max() <= 1e-10, err[ok].max()
            assert (np.abs(rho - rho_o) <= 1e-8 * rho_o + 64 * kap * 1.1e-16).all()
        else:
            bound, _ = weighted_bound(p, case.S, J, w, params, Yo, rho_o)
            assert (err <= bound).all(), (err.max(), bound.min())
        print(f"{name} weighted, mode {mode}: {len(J)} distinct rows of {p.s} draws, "
              f"max rel err y {err.max():.2e}")


def test_residual_band_at_sampling_point():
    case = Case("diffusion_2d", rows="random", N=16, r=8, s=64, m=2)
    p = case.prob
    S_d, blocks = device_inputs(case)
    B = np.asarray(problem.full_matrix(p, p.sel_param) @ case.S)
    eps = leverage.band_epsilon(p.r, p.s)
    rng = np.random.default_rng(3)
    inside, trials = 0, 24
    P = torch.from_numpy(np.ascontiguousarray(p.sel_param[None, :])).cuda()
    for _ in range(trials):
        J, w, _ = leverage_rows(p, S_d, blocks, p.sel_param, p.s, rng.uniform(size=p.s))
        sv = AffineSolver(p, None, J, mode=api.SAS_MODE_PLAIN, S_device=S_d, blocks_device=blocks,
                          weights=w)
        Y = torch.empty((1, p.r), dtype=torch.float64, device="cuda")
        rho = torch.empty(1, dtype=torch.float64, device="cuda")
        sv.solve(P, api.SAS_OUT_Y, Y, None, rho)
        torch.cuda.synchronize()
        sv.close()
        y = Y.cpu().numpy()[0]
        est = rho.item() * np.linalg.norm(w * p.b[J])  # ||W (M y - b_J)||
        true = np.linalg.norm(B @ y - p.b)
        inside += (1 - eps) * true <= est <= (1 + eps) * true
    assert inside >= 0.8 * trials, inside


def test_scores_survive_a_numerically_dependent_rhs():
    """p_sel at a snapshot point: b = A(p_sel) x(p_sel) lies in span(A(p_sel) S) to
    rounding, so [A(p_sel) S, b] has a singular value near u; the shifted first pass
    keeps the factorisation defined and the scores still sum to r + 1."""
    case = Case("diffusion_2d", rows="random", N=20, r=8, s=40, m=4)
    p = case.prob
    S_d, blocks = device_inputs(case)
    u = np.random.default_rng(4).uniform(size=p.s)
    J, w, scores = leverage_rows(p, S_d, blocks, p.snap_params[3], p.s, u)
    assert np.isfinite(scores).all() and (scores >= 0).all()
    assert abs(scores.sum() - (p.r + 1)) < 1e-6 * (p.r + 1)
