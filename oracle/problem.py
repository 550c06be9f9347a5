"""Operator families of the oracle: theta(p), explicit rows of A(p), full A(p).

The affine form A(p) = sum_k theta_k(p) A_k follows the paper's remark that
S A(p) X can be formed from precomputed pieces when A(p) varies in a
structured way (Sec. 3.1, "Computing S A(p*) X"; the transfer-function form
A(p) = pE - A_0 of Sec. 5.2).  The oracle never uses that shortcut for the
answer: it forms the s explicit rows of A(p) (Alg. 1 step 4) and multiplies
them by S.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def theta(rule: str, p) -> np.ndarray:
    """Coefficients theta_k(p) of A(p) = sum_k theta_k(p) A_k.

    "linear": (1, p_1, ..., p_d).  "pencil": A(s) = s E - A_0 at s = i*omega,
    so theta = (-1, i*omega) against the blocks (A_0, E).  "delay": the delay
    system of Sec. 5.2.3, A(p) = p I - A_0 - e^{tau p} A_1 at p = i*omega, with
    the parameter vector (omega, tau): theta = (i omega, -1, -e^{i omega tau})
    against the blocks (I, A_0, A_1).
    """
    p = np.atleast_1d(np.asarray(p, dtype=np.float64))
    if rule == "linear":
        return np.concatenate([[1.0], p])
    if rule == "pencil":
        return np.array([-1.0 + 0j, 1j * p[0]])
    if rule == "delay":
        return np.array([1j * p[0], -1.0 + 0j, -np.exp(1j * p[0] * p[1])])
    raise ValueError(f"unknown theta rule {rule!r}")


def full_matrix(prob, p) -> sp.csr_matrix:
    """A(p) as a sparse matrix (used for direct solves and true residuals)."""
    th = theta(prob.theta_rule, p)
    A = th[0] * prob.blocks[0]
    for k in range(1, len(prob.blocks)):
        A = A + th[k] * prob.blocks[k]
    return A.tocsr()


def rows(prob, p, J) -> sp.csr_matrix:
    """The s rows A(p)_{J,:} formed row by row from the operator definition."""
    th = theta(prob.theta_rule, p)
    J = np.asarray(J)
    R = th[0] * prob.blocks[0][J, :]
    for k in range(1, len(prob.blocks)):
        R = R + th[k] * prob.blocks[k][J, :]
    return R.tocsr()
