"""Finite-difference and kernel operators of the five synthetic workloads.

Every matrix is returned as scipy.sparse CSR in float64.  Index order is
lexicographic with the first grid coordinate fastest (u[i + N*j] for 2-D,
u[i + N*j + N*N*k] for 3-D).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tridiag_laplacian(n: int) -> sp.csr_matrix:
    """Unscaled 1-D Laplacian: 2 on the diagonal, -1 on both off-diagonals."""
    main = np.full(n, 2.0)
    off = np.full(n - 1, -1.0)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr")


def diffusion_2d(N: int, a_xface: np.ndarray, a_yface: np.ndarray, h: float) -> sp.csr_matrix:
    """5-point discretisation of -div(a grad u) on an N x N interior grid.

    ``a_xface[i, j]`` is the coefficient on the x-face between interior
    columns i-1 and i (i = 0..N, shape (N+1, N)); ``a_yface[i, j]`` the
    coefficient on the y-face between rows j-1 and j (shape (N, N+1)).
    Dirichlet boundary: faces touching the boundary still contribute their
    coefficient to the diagonal.  Scaled by 1/h^2.  Built row by row in CSR
    order (south, west, centre, east, north), so no sorting is needed.
    """
    n = N * N
    aw = a_xface[:-1, :].ravel(order="F")   # face west of node (i, j), node index i + N j
    ae = a_xface[1:, :].ravel(order="F")
    as_ = a_yface[:, :-1].ravel(order="F")
    an = a_yface[:, 1:].ravel(order="F")
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = idx // N
    cols = np.stack([idx - N, idx - 1, idx, idx + 1, idx + N], axis=1)
    vals = np.stack([-as_, -aw, aw + ae + as_ + an, -ae, -an], axis=1) / (h * h)
    valid = np.stack([j > 0, i > 0, np.ones(n, dtype=bool), i < N - 1, j < N - 1], axis=1)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(valid.sum(axis=1), out=indptr[1:])
    A = sp.csr_matrix((vals[valid], cols[valid].astype(np.int32), indptr), shape=(n, n))
    A.has_sorted_indices = True
    return A


def gaussian_bump_faces(N: int, centre: np.ndarray, width: float):
    """Bump psi(x) = exp(-|x - c|^2 / (2 w^2)) sampled exactly at face midpoints.

    Interior node (i, j) sits at ((i+1) h, (j+1) h), h = 1/(N+1).  The x-face
    between columns i-1 and i sits at ((i + 1/2) h, (j+1) h), i = 0..N.
    """
    h = 1.0 / (N + 1)
    xf = (np.arange(N + 1) + 0.5) * h
    xn = (np.arange(N) + 1.0) * h
    cx, cy = float(centre[0]), float(centre[1])
    gx = np.exp(-((xf - cx) ** 2) / (2 * width * width))
    gy = np.exp(-((xn - cy) ** 2) / (2 * width * width))
    a_x = np.outer(gx, gy)  # (N+1, N): x-faces
    gx_n = np.exp(-((xn - cx) ** 2) / (2 * width * width))
    gy_f = np.exp(-((xf - cy) ** 2) / (2 * width * width))
    a_y = np.outer(gx_n, gy_f)  # (N, N+1): y-faces
    return a_x, a_y


def delay_blocks(n: int, tau: float, kappa: float):
    """(I, A_0, A_1) of the delay system: A_1 = (T - kappa I) / tau, A_0 = 3 A_1, where T
    is tridiagonal with ones on both off-diagonals and T_11 = T_nn = 1 (Sec. 5.2.3)."""
    off = np.ones(n - 1)
    diag = np.zeros(n)
    diag[0] = diag[-1] = 1.0
    T = sp.diags([off, diag, off], [-1, 0, 1], format="csr")
    A1 = ((T - kappa * sp.identity(n, format="csr")) / tau).tocsr()
    A0 = (3.0 * A1).tocsr()
    return sp.identity(n, format="csr", dtype=np.float64), A0, A1


def heat_3d(N: int) -> sp.csr_matrix:
    """A0 = h^-2 * (7-point Laplacian), -6 on the diagonal, +1 on neighbours.

    Dirichlet boundary on an N^3 interior grid, h = 1/(N+1).  -A0 is SPD.
    """
    h = 1.0 / (N + 1)
    T = sp.diags([np.ones(N - 1), np.full(N, -2.0), np.ones(N - 1)], [-1, 0, 1], format="csr")
    I = sp.identity(N, format="csr")
    A = sp.kron(I, sp.kron(I, T)) + sp.kron(I, sp.kron(T, I)) + sp.kron(T, sp.kron(I, I))
    A = A.tocsr()
    A.sort_indices()
    return (A / (h * h)).tocsr()


def gaussian_kernel_block(Xa: np.ndarray, Xb: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian kernel exp(-|x - x'|^2 / (2 sigma^2)) between two point sets.

    Used only to build small dense KRR systems for snapshot generation.
    """
    d2 = ((Xa[:, None, :] - Xb[None, :, :]) ** 2).sum(-1)
    return np.exp(-d2 / (2.0 * sigma * sigma))
