"""Pins of the oracle's offline steps (Alg. 1 steps 1-2): snapshots and thin QR."""
import numpy as np

from oracle import problem, snapshots
from workloads import get_config


def test_thin_qr_hand_example():
    # Gram-Schmidt by hand: q1 = x1 / 5, R12 = q1 . x2 = 2.2, x2 - 2.2 q1 = (-0.32, 0.24, 2)
    X = np.array([[3.0, 1.0], [4.0, 2.0], [0.0, 2.0]])
    Q, R = snapshots.thin_qr(X)
    r22 = np.sqrt(0.32 ** 2 + 0.24 ** 2 + 4.0)
    np.testing.assert_allclose(R, [[5.0, 2.2], [0.0, r22]], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(Q[:, 0], [0.6, 0.8, 0.0], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(Q[:, 1], np.array([-0.32, 0.24, 2.0]) / r22, rtol=1e-14, atol=1e-15)
    # a negative column keeps R_11 > 0 and flips q1
    Q2, R2 = snapshots.thin_qr(-X)
    np.testing.assert_allclose(R2, R, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(Q2, -Q, rtol=1e-14, atol=1e-15)


def test_thin_qr_complex_properties():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((50, 7)) + 1j * rng.standard_normal((50, 7))
    Q, R = snapshots.thin_qr(X)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(7), atol=1e-14)
    np.testing.assert_allclose(Q @ R, X, atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0)
    d = np.diag(R)
    assert (np.abs(d.imag) == 0).all() and (d.real > 0).all()
    # uniqueness: an independent Gram-Schmidt gives the same factors
    Qg = np.zeros_like(X)
    for j in range(7):
        v = X[:, j].copy()
        for _ in range(2):
            v -= Qg[:, :j] @ (Qg[:, :j].conj().T @ v)
        Qg[:, j] = v / np.linalg.norm(v)
    np.testing.assert_allclose(Q, Qg, atol=1e-13)


def test_snapshot_solves_satisfy_the_system():
    for name, kw in [("diffusion_2d", dict(N=16, r=6, s=12, m=4)),
                     ("transfer_function", dict(N=5, r=4, s=8, m=4)),
                     ("delay_system", dict(n=400, r=5, s=10, m=4))]:
        prob = get_config(name, **kw)
        X = snapshots.snapshot_matrix(prob)
        for j, p in enumerate(prob.snap_params):
            A = problem.full_matrix(prob, p)
            res = np.linalg.norm(A @ X[:, j] - prob.b) / np.linalg.norm(prob.b)
            assert res < 1e-12, (name, j, res)
