"""Pins of the oracle's leverage-score sampling and residual estimate (Sec. 4.3.2-4.3.3).

Each check ties the oracle to something other than itself:
  * the scores equal the diagonal of the hat matrix V (V^H V)^{-1} V^H (the
    textbook definition, not the QR the oracle uses), sum to the rank, and
    depend on span(V) only;
  * inverse-CDF sampling against a hand-worked draw;
  * the weighted sketch is unbiased, E ||S r||^2 = ||r||^2 (Monte Carlo);
  * weighted least squares over every row with unit weights is the full
    least-squares problem (ApSnap);
  * at the sampling parameter the weighted subsampled residual brackets the true
    residual within (1 -/+ eps) in most draws (Sec. 4.3.3).
"""
import numpy as np
import pytest

from oracle import leverage, online, problem
from workloads import get_config
from workloads import snapshots as wsnap


@pytest.mark.parametrize("cplx", [False, True])
def test_scores_are_the_hat_matrix_diagonal(cplx):
    rng = np.random.default_rng(3)
    V = rng.standard_normal((40, 5)) + (1j * rng.standard_normal((40, 5)) if cplx else 0)
    H = V @ np.linalg.inv(V.conj().T @ V) @ V.conj().T
    lev = leverage.leverage_scores(V)
    np.testing.assert_allclose(lev, np.real(np.diag(H)), rtol=1e-12, atol=1e-14)
    assert abs(lev.sum() - 5) < 1e-12
    assert (lev >= -1e-15).all() and (lev <= 1 + 1e-12).all()
    X = rng.standard_normal((5, 5)) + 3 * np.eye(5)
    np.testing.assert_allclose(leverage.leverage_scores(V @ X), lev, rtol=1e-10, atol=1e-13)


def test_orthonormal_columns_give_row_norms():
    Q, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((30, 4)))
    np.testing.assert_allclose(leverage.leverage_scores(Q), (Q * Q).sum(1), rtol=1e-12)


def test_inverse_cdf_draws_by_hand():
    # pi = (0.1, 0.3, 0.6): cdf (0.1, 0.4, 1.0); u = 0.05 -> 0, 0.1 -> 1 (cdf > u strictly),
    # 0.39 -> 1, 0.4 -> 2, 0.99 -> 2
    scores = np.array([0.5, 1.5, 3.0])
    J, w = leverage.sample_rows(scores, 5, np.array([0.05, 0.1, 0.39, 0.4, 0.99]))
    np.testing.assert_array_equal(J, [0, 1, 2])
    np.testing.assert_allclose(w, np.sqrt(np.array([1, 2, 2]) / (5 * np.array([0.1, 0.3, 0.6]))))


def test_weighted_sketch_is_unbiased():
    rng = np.random.default_rng(5)
    n, s = 200, 20
    scores = rng.uniform(0.1, 1.0, n)
    res = rng.standard_normal(n)
    vals = []
    for t in range(4000):
        J, w = leverage.sample_rows(scores, s, rng.uniform(size=s))
        vals.append(np.sum((w * res[J]) ** 2))
    vals = np.array(vals)
    se = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - np.sum(res ** 2)) <= 4 * se


def test_all_rows_unit_weights_is_apsnap():
    prob = get_config("reaction_diffusion_1d", n=200, r=6, s=12, m=3)
    S = wsnap.basis(prob)
    J = np.arange(prob.n)
    for p in prob.test_params:
        y, _ = online.solve_one(prob, S, J, p, w=np.ones(prob.n))
        B = problem.full_matrix(prob, p).toarray() @ S
        ref = np.linalg.lstsq(B, prob.b, rcond=None)[0]
        np.testing.assert_allclose(y, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_band_brackets_true_residual_at_sampling_point():
    prob = get_config("diffusion_2d", N=16, r=8, s=64, m=2)
    S = wsnap.basis(prob)
    p = prob.sel_param
    B = np.asarray(problem.full_matrix(prob, p) @ S)
    lev = leverage.leverage_scores(np.column_stack([B, prob.b]))
    eps = leverage.band_epsilon(prob.r, prob.s)
    rng = np.random.default_rng(6)
    inside = 0
    trials = 60
    for _ in range(trials):
        J, w = leverage.sample_rows(lev, prob.s, rng.uniform(size=prob.s))
        y, _ = online.solve_one(prob, S, J, p, w=w)
        est = np.linalg.norm(w * (B[J] @ y - prob.b[J]))
        true = np.linalg.norm(B @ y - prob.b)
        inside += (1 - eps) * true <= est <= (1 + eps) * true
    assert inside >= 0.9 * trials
