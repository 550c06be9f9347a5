"""The seeded workload generators: operators against their definitions, snapshot solvers."""
import numpy as np
import pytest

from workloads import get_config, operators as ops, snapshots as wsnap


def test_diffusion_stencil_matches_definition():
    N, h = 7, 1.0 / 8
    ax = np.random.default_rng(0).uniform(1, 2, (N + 1, N))
    ay = np.random.default_rng(1).uniform(1, 2, (N, N + 1))
    A = ops.diffusion_2d(N, ax, ay, h).toarray()
    B = np.zeros((N * N, N * N))
    for j in range(N):
        for i in range(N):
            r = i + N * j
            B[r, r] = (ax[i, j] + ax[i + 1, j] + ay[i, j] + ay[i, j + 1]) / h ** 2
            if i > 0:
                B[r, r - 1] = -ax[i, j] / h ** 2
            if i < N - 1:
                B[r, r + 1] = -ax[i + 1, j] / h ** 2
            if j > 0:
                B[r, r - N] = -ay[i, j] / h ** 2
            if j < N - 1:
                B[r, r + N] = -ay[i, j + 1] / h ** 2
    np.testing.assert_array_equal(A, B)
    # constant coefficient: symmetric positive definite with the known smallest eigenvalue
    L = ops.diffusion_2d(N, np.ones((N + 1, N)), np.ones((N, N + 1)), h).toarray()
    lam = np.linalg.eigvalsh(L)
    np.testing.assert_allclose(lam[0], 8 * np.sin(np.pi * h / 2) ** 2 / h ** 2, rtol=1e-12)


def test_heat_3d_is_negative_laplacian():
    A = ops.heat_3d(4).toarray()
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).max() < 0


def test_diffusion_pcg_matches_direct():
    prob = get_config("diffusion_2d", N=24, r=4, m=2)
    X, res = wsnap.diffusion_pcg(prob, prob.snap_params, device="cpu", rtol=1e-12)
    Xd = wsnap.snapshot_solutions(prob)
    assert res.max() < 1e-11
    np.testing.assert_allclose(X.numpy().T, Xd, rtol=1e-9, atol=1e-12 * np.abs(Xd).max())


def test_transfer_cocg_matches_direct():
    prob = get_config("transfer_function", N=6, r=5, m=2)
    X, res = wsnap.transfer_cocg(prob, prob.snap_params[:, 0], device="cpu", rtol=1e-12)
    Xd = wsnap.snapshot_solutions(prob)
    np.testing.assert_allclose(X.numpy().T, Xd, rtol=1e-8, atol=1e-12 * np.abs(Xd).max())


def test_gram_schmidt_twice_is_orthonormal():
    torch = pytest.importorskip("torch")
    X = torch.randn(300, 12, dtype=torch.float64)
    Q = wsnap.orthonormalise_torch(X)
    assert torch.linalg.vector_norm(Q.T @ Q - torch.eye(12)) < 1e-13
    P = Q @ Q.T
    assert torch.linalg.vector_norm(P @ X - X) < 1e-10 * torch.linalg.vector_norm(X)
