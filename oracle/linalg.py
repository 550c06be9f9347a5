"""Small dense and banded solvers of the oracle."""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def thomas(lower: np.ndarray, diag: np.ndarray, upper: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Tridiagonal solve by forward elimination and back substitution.

    ``lower[i]`` multiplies x[i-1] in row i (lower[0] unused), ``upper[i]``
    multiplies x[i+1] (upper[n-1] unused).  ``diag`` and ``rhs`` may carry a
    trailing batch axis, so many systems with the same band pattern are
    solved at once (row index first).
    """
    n = diag.shape[0]
    dt = np.result_type(diag, rhs, upper, lower)
    c = np.empty(diag.shape, dtype=dt)
    d = np.empty(np.broadcast_shapes(diag.shape, rhs.shape), dtype=dt)
    c[0] = upper[0] / diag[0]
    d[0] = rhs[0] / diag[0]
    for i in range(1, n):
        den = diag[i] - lower[i] * c[i - 1]
        if i < n - 1:
            c[i] = upper[i] / den
        d[i] = (rhs[i] - lower[i] * d[i - 1]) / den
    x = np.empty_like(d)
    x[n - 1] = d[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = d[i] - c[i] * x[i + 1]
    return x


def least_squares(M: np.ndarray, rhs: np.ndarray):
    """argmin_y ||M y - rhs||_2 for full-column-rank M (s >= r), Householder QR.

    Returns (y, rho) with rho = ||M y - rhs||_2 taken from the part of Q^H rhs
    that the triangular solve does not use (the s - r trailing components of
    the full Q^H rhs), which is the least-squares residual norm.
    """
    s, r = M.shape
    Q, R = np.linalg.qr(M, mode="complete")
    z = Q.conj().T @ rhs
    y = sla.solve_triangular(R[:r, :r], z[:r], lower=False)
    rho = float(np.linalg.norm(z[r:])) if s > r else 0.0
    return y, rho
