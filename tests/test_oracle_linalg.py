"""Pins of the oracle's small solvers against closed forms and brute force."""
import os

import mpmath
import numpy as np
import pytest

from oracle import linalg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    M, vals = [], {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        key, *nums = line.split()
        if key == "M":
            M.append([float(v) for v in nums])
        else:
            vals[key] = np.array([float(v) for v in nums])
    return np.array(M), vals


def test_least_squares_hand_example():
    M, v = _read_golden("ls_hand.txt")
    y, rho = linalg.least_squares(M, v["b"])
    np.testing.assert_allclose(y, v["y"], rtol=1e-15, atol=1e-15)
    assert abs(rho - v["res"][0]) < 1e-15


@pytest.mark.parametrize("cplx", [False, True])
def test_least_squares_extended_precision(cplx):
    """Brute force: normal equations solved with 60 significant digits."""
    rng = np.random.default_rng(1)
    s, r = 9, 4
    M = rng.standard_normal((s, r))
    b = rng.standard_normal(s)
    if cplx:
        M = M + 1j * rng.standard_normal((s, r))
        b = b + 1j * rng.standard_normal(s)
    y, rho = linalg.least_squares(M, b)
    mpmath.mp.dps = 60
    Mm = mpmath.matrix([[mpmath.mpc(complex(M[i, j])) for j in range(r)] for i in range(s)])
    bm = mpmath.matrix([mpmath.mpc(complex(b[i])) for i in range(s)])
    MH = Mm.transpose_conj()
    ym = mpmath.lu_solve(MH * Mm, MH * bm)
    yref = np.array([complex(ym[i]) for i in range(r)])
    if not cplx:
        yref = yref.real
    assert np.linalg.norm(y - yref) / np.linalg.norm(yref) < 1e-13
    res = Mm * ym - bm
    rho_ref = float(mpmath.norm(res))
    assert abs(rho - rho_ref) / rho_ref < 1e-12


def test_least_squares_residual_is_orthogonal():
    """Normal-equation optimality: M^T (b - M y) = 0 up to rounding."""
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 20))
    b = rng.standard_normal(40)
    y, rho = linalg.least_squares(M, b)
    r = b - M @ y
    assert np.linalg.norm(M.T @ r) < 1e-12 * np.linalg.norm(M) * np.linalg.norm(b)
    assert abs(np.linalg.norm(r) - rho) < 1e-12


def test_thomas_matches_dense_solve():
    rng = np.random.default_rng(3)
    n = 50
    lower = np.concatenate([[0.0], rng.standard_normal(n - 1)])
    upper = np.concatenate([rng.standard_normal(n - 1), [0.0]])
    diag = 4.0 + rng.uniform(0, 1, n)
    rhs = rng.standard_normal(n)
    A = np.diag(diag) + np.diag(lower[1:], -1) + np.diag(upper[:-1], 1)
    x = linalg.thomas(lower, diag, upper, rhs)
    np.testing.assert_allclose(A @ x, rhs, atol=1e-13)
    # batched diagonals, shared right-hand side
    diags = diag[:, None] + np.arange(3)[None, :]
    X = linalg.thomas(lower, diags, upper, rhs[:, None])
    for k in range(3):
        Ak = A + k * np.eye(n)
        np.testing.assert_allclose(Ak @ X[:, k], rhs, atol=1e-13)
