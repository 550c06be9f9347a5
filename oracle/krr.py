"""Kernel ridge regression rows in the oracle (Sec. 5.3).

A(sigma, lambda) = K_sigma + lambda I with K_ij = exp(-|x_i - x_j|^2 / (2 sigma^2))
(Eq. for K in Sec. 5.3).  Only the s rows at J are formed, from direct
coordinate differences, so M = K_sigma(X_J, X) S + lambda S_J.
"""
from __future__ import annotations

import numpy as np

from . import linalg


def kernel_rows(X: np.ndarray, J, sigma: float, chunk: int = 65536) -> np.ndarray:
    """K_sigma(X_J, X): s x N kernel entries from direct differences."""
    J = np.asarray(J)
    XJ = X[J]
    out = np.empty((len(J), X.shape[0]))
    for a in range(0, X.shape[0], chunk):
        B = X[a:a + chunk]
        d2 = np.zeros((len(J), B.shape[0]))
        for k in range(X.shape[1]):
            diff = XJ[:, k][:, None] - B[:, k][None, :]
            d2 += diff * diff
        out[:, a:a + chunk] = np.exp(-d2 / (2.0 * sigma * sigma))
    return out


def subsampled_matrix(X, S, J, p) -> np.ndarray:
    sigma, lam = float(p[0]), float(p[1])
    J = np.asarray(J)
    return kernel_rows(X, J, sigma) @ S + lam * S[J]


def full_matrix(X, p) -> np.ndarray:
    """Dense K_sigma + lambda I (small N only)."""
    sigma, lam = float(p[0]), float(p[1])
    K = kernel_rows(X, np.arange(X.shape[0]), sigma)
    return K + lam * np.eye(X.shape[0])


def solve_one(prob, S, J, p):
    J = np.asarray(J)
    M = subsampled_matrix(prob.X, S, J, p)
    bJ = prob.b[J]
    y, res = linalg.least_squares(M, bJ)
    return y, res / np.linalg.norm(bJ)


def solve_many(prob, S, J, params):
    ys, rhos = [], []
    for p in params:
        y, rho = solve_one(prob, S, J, p)
        ys.append(y)
        rhos.append(rho)
    return np.array(ys), np.array(rhos)


def snapshot_matrix(prob) -> np.ndarray:
    """Direct dense solves (K_sigma + lambda I) x = y at the snapshot grid (small N)."""
    cols = [np.linalg.solve(full_matrix(prob.X, p), prob.b) for p in prob.snap_params]
    return np.stack(cols, axis=1)


def true_residual(prob, p, x) -> float:
    A = full_matrix(prob.X, p)
    return float(np.linalg.norm(A @ x - prob.b) / np.linalg.norm(prob.b))
