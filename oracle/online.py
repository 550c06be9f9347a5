"""Online stage of SubApSnap in the oracle (Alg. 1 step 4; Sec. 3; Sec. 5.2.2).

For each new parameter p:
  M(p)  = (A(p)_{J,:}) S          explicit rows of A(p) times the basis
  y     = argmin ||M(p) y - b_J||   small s x r least squares
  x_hat = S y                     reconstruction, or
  H     = (c^T S) y               quantity of interest without any n-vector
The subsampled relative residual ||M y - b_J|| / ||b_J|| is the online
estimate of the true residual (Sec. 4.3.1); the true residual
||A(p) x_hat - b|| / ||b|| is what Tables 3-4 report as (max, median).
"""
from __future__ import annotations

import numpy as np

from . import linalg, problem


def subsampled_matrix(prob, S: np.ndarray, J, p) -> np.ndarray:
    """M(p) = A(p)_{J,:} S from the explicit rows (Alg. 1 step 4)."""
    R = problem.rows(prob, p, J)
    return np.asarray(R @ S)


def solve_one(prob, S, J, p, bJ=None, w=None):
    """(y, rho_sub): subsampled LS solution and its relative residual.

    With row weights w (leverage-score sampling, Sec. 4.3.2 footnote) the rows
    of M and b_J are scaled by w: y = argmin ||W (M y - b_J)||, and rho is
    ||W (M y - b_J)|| / ||W b_J||.
    """
    J = np.asarray(J)
    if bJ is None:
        bJ = prob.b[J]
    M = subsampled_matrix(prob, S, J, p)
    if w is not None:
        M = M * np.asarray(w)[:, None]
        bJ = bJ * np.asarray(w)
    y, res = linalg.least_squares(M, bJ)
    return y, res / np.linalg.norm(bJ)


def solve_many(prob, S, J, params, w=None):
    """Y (m x r) and rho_sub (m) for a list of parameters."""
    ys, rhos = [], []
    for p in params:
        y, rho = solve_one(prob, S, J, p, w=w)
        ys.append(y)
        rhos.append(rho)
    return np.array(ys), np.array(rhos)


def reconstruct(S: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """x_hat = S y for every row of Y; returns (m, n)."""
    return (S @ Y.T).T


def qoi_vector(prob, S: np.ndarray) -> np.ndarray:
    """The r-vector c^T S (Sec. 5.2.2: precompute c^T X; plain transpose)."""
    if prob.qoi_kind == "mean":
        return S.sum(axis=0) / prob.n
    return prob.c @ S


def qoi(prob, S, Y) -> np.ndarray:
    """H(p) ~ (c^T S) y for every row of Y."""
    return Y @ qoi_vector(prob, S)


def true_residual(prob, p, x: np.ndarray) -> float:
    """||A(p) x - b|| / ||b|| with the full operator."""
    A = problem.full_matrix(prob, p)
    return float(np.linalg.norm(A @ x - prob.b) / np.linalg.norm(prob.b))


def subsampled_residual(prob, S, J, p, y) -> float:
    """||M(p) y - b_J|| / ||b_J|| for a given coefficient vector y."""
    J = np.asarray(J)
    M = subsampled_matrix(prob, S, J, p)
    bJ = prob.b[J]
    return float(np.linalg.norm(M @ y - bJ) / np.linalg.norm(bJ))


def condition_number(prob, S, J, p) -> float:
    """2-norm condition number of M(p) (used to scale parity tolerances)."""
    M = subsampled_matrix(prob, S, J, p)
    sv = np.linalg.svd(M, compute_uv=False)
    return float(sv[0] / sv[-1])
