"""Offline steps 1-2 of Algorithm 1 in the oracle: snapshots and basis.

Step 1 solves A(p_i) x(p_i) = b at the r snapshot parameters; step 2 replaces
X by the Q factor of its thin QR (Sec. 3.1, "Postprocessing the snapshot
matrix X"), which leaves the online answer unchanged.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import linalg, problem


def solve_full(prob, p) -> np.ndarray:
    """Direct solve of A(p) x = b (Thomas for tridiagonal, sparse LU otherwise)."""
    A = problem.full_matrix(prob, p)
    if prob.name == "reaction_diffusion_1d":
        diag = A.diagonal()
        lower = np.concatenate([[0.0], A.diagonal(-1)])
        upper = np.concatenate([A.diagonal(1), [0.0]])
        return linalg.thomas(lower, diag, upper, prob.b)
    return spla.spsolve(A.tocsc(), prob.b)


def solve_full_batch_1d(prob, params: np.ndarray) -> np.ndarray:
    """Thomas solves of the 1-D reaction-diffusion system for many p at once.

    A(p) = L + p D has the band (-1, 2 + p d_i, -1); returns x as (m, n).
    """
    d = prob.meta["d"]
    n = prob.n
    ps = np.asarray(params, dtype=np.float64).reshape(-1)
    diag = 2.0 + d[:, None] * ps[None, :]
    lower = np.full(n, -1.0); lower[0] = 0.0
    upper = np.full(n, -1.0); upper[-1] = 0.0
    x = linalg.thomas(lower, diag, upper, prob.b[:, None])
    return x.T.copy()


def snapshot_matrix(prob) -> np.ndarray:
    """X = [x(p_1), ..., x(p_r)] from direct solves (Alg. 1 step 1)."""
    if prob.name == "reaction_diffusion_1d":
        return solve_full_batch_1d(prob, prob.snap_params[:, 0]).T.copy()
    cols = [solve_full(prob, p) for p in prob.snap_params]
    return np.stack(cols, axis=1)


def orthonormal_basis(X: np.ndarray) -> np.ndarray:
    """Thin-QR Q factor of the snapshot matrix (Alg. 1 step 2)."""
    Q, _ = np.linalg.qr(X, mode="reduced")
    return Q


def thin_qr(X: np.ndarray):
    """Thin QR X = Q R with R's diagonal real and non-negative (Alg. 1 step 2).

    LAPACK's Householder QR, then each column j of Q multiplied by the phase
    of R_jj and row j of R by its conjugate, which leaves Q R unchanged and
    makes the factorisation unique when X has full column rank.
    """
    Q, R = np.linalg.qr(np.asarray(X), mode="reduced")
    d = np.diag(R).copy()
    mag = np.abs(d)
    ph = np.where(mag > 0, d / np.where(mag > 0, mag, 1.0), 1.0)
    Q = Q * ph[None, :]
    R = np.conj(ph)[:, None] * R
    return Q, R
