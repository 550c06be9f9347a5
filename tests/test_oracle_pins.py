"""Pins of the oracle's online stage against what the paper fixes.

(i)   s = n: SubApSnap is ApSnap, the full least squares on A(p) S (Sec. 3, Eq. 2).
(ii)  p equal to a snapshot parameter: x_hat = x(p) (Sec. 4.2 example: the
      residual is zero at the snapshot points by construction).
(iii) s = r: interpolation, (A(p) x_hat)_J = b_J (Sec. 3).
(iv)  A = I: SubSnap = DEIM, x_hat = S (S_J)^+ b_J (Sec. 3.4).
(v)   Lemma 4.1 (a)-(c) on random instances.
(vi)  Invariances: S -> S Q (Sec. 3.1) and permutations of J.
(vii) CPQR round 1 equals LAPACK's pivoted QR where there are no near-ties.
A nonsymmetric operator family is included so that a transposed operand
cannot hide behind symmetric test matrices.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import krr, linalg, online, problem, selection, snapshots
from workloads import get_config
from workloads.configs import AffineProblem


def nonsymmetric_problem(n=30, r=5, s=9, seed=7, cplx=False):
    rng = np.random.default_rng(seed)
    A0 = sp.random(n, n, density=0.2, random_state=rng) + sp.diags(np.full(n, 5.0))
    A1 = sp.random(n, n, density=0.2, random_state=rng)
    b = rng.standard_normal(n)
    return AffineProblem(
        name="nonsym", n=n, blocks=[A0.tocsr(), A1.tocsr()],
        theta_rule="pencil" if cplx else "linear",
        b=b.astype(np.complex128) if cplx else b, r=r, s=s,
        snap_params=np.linspace(0.0, 1.0, r)[:, None], sel_param=np.array([0.5]),
        test_params=rng.uniform(0, 1, (6, 1)), complex_valued=cplx,
    )


def basis_and_rows(prob):
    X = snapshots.snapshot_matrix(prob)
    S = snapshots.orthonormal_basis(X)
    V = np.asarray(problem.full_matrix(prob, prob.sel_param) @ S)
    J, gaps = selection.cpqr_rows(V, prob.s)
    return X, S, J


@pytest.mark.parametrize("cplx", [False, True])
def test_full_sampling_is_apsnap(cplx):
    prob = nonsymmetric_problem(cplx=cplx)
    X, S, _ = basis_and_rows(prob)
    J = np.arange(prob.n)
    for p in prob.test_params:
        y, _ = online.solve_one(prob, S, J, p)
        B = problem.full_matrix(prob, p).toarray() @ S
        c_ref = np.linalg.lstsq(B, prob.b, rcond=None)[0]  # SVD-based solver
        assert np.linalg.norm(y - c_ref) <= 1e-12 * np.linalg.norm(c_ref)


@pytest.mark.parametrize("name,kw", [
    ("nonsym", {}),
    ("reaction_diffusion_1d", dict(n=256, r=8, s=16, m=4)),
    ("diffusion_2d", dict(N=12, r=6, s=12, m=4)),
    ("transfer_function", dict(N=5, r=5, s=12, m=4)),
    ("delay_system", dict(n=300, r=8, s=16, m=4)),
])
def test_snapshot_parameter_recovers_solution(name, kw):
    prob = nonsymmetric_problem() if name == "nonsym" else get_config(name, **kw)
    X, S, J = basis_and_rows(prob)
    for i in (0, prob.r // 2, prob.r - 1):
        p = prob.snap_params[i]
        y, rho = online.solve_one(prob, S, J, p)
        xh = S @ y
        x = X[:, i]
        kappa = online.condition_number(prob, S, J, p)
        assert np.linalg.norm(xh - x) <= 1e-14 * kappa * np.linalg.norm(x) + 1e-300
        assert rho <= 1e-13 * kappa


@pytest.mark.parametrize("cplx", [False, True])
def test_square_subsample_interpolates(cplx):
    prob = nonsymmetric_problem(cplx=cplx)
    prob.s = prob.r
    X, S, J = basis_and_rows(prob)
    assert len(J) == prob.r
    for p in prob.test_params:
        y, rho = online.solve_one(prob, S, J, p)
        Ax = problem.full_matrix(prob, p) @ (S @ y)
        np.testing.assert_allclose(Ax[J], prob.b[J], atol=1e-11 * np.abs(prob.b).max())
        assert rho < 1e-12


@pytest.mark.parametrize("s", [6, 10])
def test_identity_operator_is_deim(s):
    rng = np.random.default_rng(11)
    n, r = 40, 6
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    yvec = U @ rng.standard_normal(r) + 1e-3 * rng.standard_normal(n)
    prob = AffineProblem(name="deim", n=n, blocks=[sp.identity(n, format="csr")], theta_rule="linear",
                         b=yvec, r=r, s=s, snap_params=np.zeros((r, 0)), sel_param=np.zeros(0),
                         test_params=np.zeros((1, 0)))
    J, _ = selection.cpqr_rows(U, s)
    y, _ = online.solve_one(prob, U, J, np.zeros(0))
    UJ = U[J]
    if s == r:
        ref = np.linalg.solve(UJ, yvec[J])  # classical DEIM interpolation
    else:
        ref = np.linalg.pinv(UJ) @ yvec[J]  # oversampled DEIM
    np.testing.assert_allclose(U @ y, U @ ref, rtol=1e-12, atol=1e-14)


def polar_factor(B):
    W, _, Vh = np.linalg.svd(B, full_matrices=False)
    return W @ Vh


@pytest.mark.parametrize("seed", range(5))
def test_lemma_4_1_bounds(seed):
    prob = nonsymmetric_problem(seed=seed, n=40, r=5, s=8)
    X, S, J = basis_and_rows(prob)
    rng = np.random.default_rng(seed)
    for p in rng.uniform(0, 1, (4, 1)):
        B = problem.full_matrix(prob, p).toarray() @ S
        b = prob.b
        c = np.linalg.lstsq(B, b, rcond=None)[0]
        chat, _ = online.solve_one(prob, S, J, p)
        full = np.linalg.norm(B @ c - b)
        sub = np.linalg.norm(B @ chat - b)
        assert full <= sub * (1 + 1e-12)                      # (a)
        U = polar_factor(B)
        bound_b = 1.0 / np.linalg.svd(U[J], compute_uv=False)[-1]
        assert sub <= bound_b * full * (1 + 1e-10)             # (b), ||S||_2 = 1
        Ut = polar_factor(np.column_stack([B, b]))
        sv = np.linalg.svd(Ut[J], compute_uv=False)
        assert sub <= (sv[0] / sv[-1]) * full * (1 + 1e-10)   # (c)


def test_basis_rotation_and_row_order_invariance():
    prob = get_config("reaction_diffusion_1d", n=300, r=8, s=16, m=5)
    X, S, J = basis_and_rows(prob)
    Qr, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((prob.r, prob.r)))
    S2 = S @ Qr
    V2 = np.asarray(problem.full_matrix(prob, prob.sel_param) @ S2)
    J2, _ = selection.cpqr_rows(V2, prob.s)
    np.testing.assert_array_equal(J, J2)
    perm = np.random.default_rng(6).permutation(len(J))
    for p in prob.test_params:
        y1, _ = online.solve_one(prob, S, J, p)
        y2, _ = online.solve_one(prob, S2, J, p)
        y3, _ = online.solve_one(prob, S, J[perm], p)
        x1 = S @ y1
        np.testing.assert_allclose(S2 @ y2, x1, rtol=1e-9, atol=1e-12 * np.abs(x1).max())
        np.testing.assert_allclose(S @ y3, x1, rtol=1e-9, atol=1e-12 * np.abs(x1).max())


def test_cpqr_first_round_matches_lapack():
    rng = np.random.default_rng(9)
    for _ in range(5):
        V = rng.standard_normal((200, 12)) * rng.uniform(0.5, 2.0, 200)[:, None]
        J, gaps = selection.cpqr_rows(V, 12)
        _, _, piv = sla.qr(V.T, pivoting=True, mode="economic")
        assert gaps.min() > 1e-8
        np.testing.assert_array_equal(J, piv[:12])


def test_cpqr_rounds_structure():
    rng = np.random.default_rng(10)
    V = rng.standard_normal((100, 7))
    J, gaps = selection.cpqr_rows(V, 17)
    assert len(J) == 17 and len(set(J.tolist())) == 17
    # round 2 is plain CPQR on the remaining rows
    rest = np.setdiff1d(np.arange(100), J[:7])
    _, _, piv = sla.qr(V[rest].T, pivoting=True, mode="economic")
    np.testing.assert_array_equal(J[7:14], rest[piv[:7]])


def test_kernel_rows_closed_forms():
    X = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 0.0]])
    K = krr.kernel_rows(X, [0, 1], sigma=2.0)
    assert K[0, 0] == 1.0 and K[1, 1] == 1.0
    assert abs(K[0, 1] - np.exp(-25.0 / 8.0)) < 1e-16
    assert abs(K[1, 2] - np.exp(-20.0 / 8.0)) < 1e-16
    assert abs(K[0, 2] - np.exp(-1.0 / 8.0)) < 1e-16


def test_kernel_ridge_snapshot_recovery():
    prob = get_config("kernel_ridge", N=300, r=9, s=27, m=3)
    X = krr.snapshot_matrix(prob)
    S = snapshots.orthonormal_basis(X)
    V = krr.full_matrix(prob.X, prob.sel_param) @ S
    J, _ = selection.cpqr_rows(V, prob.s)
    for i in (0, 4, 8):
        p = prob.snap_params[i]
        y, rho = krr.solve_one(prob, S, J, p)
        M = krr.subsampled_matrix(prob.X, S, J, p)
        sv = np.linalg.svd(M, compute_uv=False)
        kappa = sv[0] / sv[-1]
        assert np.linalg.norm(S @ y - X[:, i]) <= 1e-14 * kappa * np.linalg.norm(X[:, i])


def test_kernel_ridge_snapshots_closed_form():
    """Two points at distance d on a line: K_sigma = [[1, e], [e, 1]] with e = exp(-d^2 / (2
    sigma^2)), so (K + lambda I) x = b has the closed form x = [(1 + lambda) b_1 - e b_2,
    (1 + lambda) b_2 - e b_1] / ((1 + lambda)^2 - e^2).  Pins full_matrix (a dropped or squared
    lambda, or sigma for sigma^2, shows) and snapshot_matrix's column order."""
    from types import SimpleNamespace
    d = 0.7
    X = np.array([[0.0], [d]])
    b = np.array([1.3, -0.4])
    grid = [(0.5, 1e-3), (0.5, 0.2), (1.7, 1e-3), (1.7, 0.2)]
    prob = SimpleNamespace(X=X, b=b, snap_params=np.array(grid))
    Xs = krr.snapshot_matrix(prob)
    for c, (sigma, lam) in enumerate(grid):
        e = np.exp(-d * d / (2.0 * sigma * sigma))
        A = krr.full_matrix(X, (sigma, lam))
        np.testing.assert_allclose(A, [[1.0 + lam, e], [e, 1.0 + lam]], rtol=0, atol=1e-16)
        det = (1.0 + lam) ** 2 - e * e
        x = np.array([(1.0 + lam) * b[0] - e * b[1], (1.0 + lam) * b[1] - e * b[0]]) / det
        np.testing.assert_allclose(Xs[:, c], x, rtol=1e-13)


def test_delay_theta_rebuilds_the_delay_operator():
    """A(p) from the delay rule and the blocks equals p I - A_0 - e^{tau p} A_1 written
    out from its definition in Sec. 5.2.3 (T tridiagonal with unit off-diagonals and
    T_11 = T_nn = 1, A_1 = (T - kappa I)/tau, A_0 = 3 A_1), at p = i omega; a swapped
    block, a sign or a missing factor tau in the exponent shows as a mismatch."""
    n, tau, kappa = 9, 0.1, 2.1
    prob = get_config("delay_system", n=n, r=4, s=8, m=3, tau=tau, kappa=kappa)
    T = np.zeros((n, n))
    for i in range(n - 1):
        T[i, i + 1] = T[i + 1, i] = 1.0
    T[0, 0] = T[-1, -1] = 1.0
    A1 = (T - kappa * np.eye(n)) / tau
    A0 = 3.0 * A1
    for omega in (0.37, 12.5, 300.0):
        p = 1j * omega
        ref = p * np.eye(n) - A0 - np.exp(tau * p) * A1
        got = problem.full_matrix(prob, np.array([omega, tau])).toarray()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_pencil_theta_rebuilds_the_transfer_function_operator():
    """A(i omega) from the pencil rule and the blocks equals i omega E - A_0 written out
    from its definition (Sec. 5.2, A(s) = s E - A_0 on the imaginary axis): A_0 the
    h^-2-scaled 7-point heat operator on an N^3 grid with zero Dirichlet values (-6 on
    the diagonal, +1 per neighbour, index i + N j + N^2 k), E = diag(e).  A sign slip
    (A_0 + i omega E), a swapped pair of blocks or a missing i fails."""
    N = 3
    prob = get_config("transfer_function", N=N, r=4, s=8, m=3)
    n, h = N ** 3, 1.0 / (N + 1)
    A0 = np.zeros((n, n))
    for k in range(N):
        for j in range(N):
            for i in range(N):
                row = i + N * j + N * N * k
                A0[row, row] = -6.0 / h ** 2
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < N and 0 <= jj < N and 0 <= kk < N:
                        A0[row, ii + N * jj + N * N * kk] = 1.0 / h ** 2
    E = np.diag(prob.meta["e"])
    for omega in (0.01, 3.0, 2500.0):
        ref = 1j * omega * E - A0
        got = problem.full_matrix(prob, np.array([omega])).toarray()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_linear_theta_rebuilds_the_diffusion_operator():
    """A(p) from the linear rule and the blocks equals -div(a(x;p) grad .) / h^2 written
    out node by node from a(x;p) = 1 + sum_k p_k psi_k(x), psi_k(x) =
    exp(-|x - c_k|^2 / (2 w^2)) evaluated at the four face midpoints of every node
    (node (i, j) at ((i+1) h, (j+1) h), index i + N j, zero Dirichlet values).  A
    dropped leading 1 (no A_0), a wrong sign on a p_k or a shifted face fails."""
    N = 5
    prob = get_config("diffusion_2d", N=N, r=4, s=8, m=3)
    h, w = prob.meta["h"], prob.meta["width"]
    centres = prob.meta["centres"]

    def a(x, y, p):
        return 1.0 + sum(pk * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / (2 * w * w))
                         for pk, c in zip(p, centres))

    rng = np.random.default_rng(5)
    for p in (np.zeros(4), np.array([1.0, 0.0, 0.0, 0.0]), rng.uniform(0, 1, 4), rng.uniform(0, 1, 4)):
        ref = np.zeros((N * N, N * N))
        for j in range(N):
            for i in range(N):
                row = i + N * j
                x, y = (i + 1) * h, (j + 1) * h
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    af = a(x + di * h / 2, y + dj * h / 2, p)
                    ref[row, row] += af / h ** 2
                    ii, jj = i + di, j + dj
                    if 0 <= ii < N and 0 <= jj < N:
                        ref[row, ii + N * jj] = -af / h ** 2
        got = problem.full_matrix(prob, p).toarray()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_qoi_hand_worked_transpose_and_mean():
    """The QoI H = c^T x_hat = (c^T S) y with the plain transpose (Sec. 5.2.2, H ~ (c^T X) c_hat;
    Sec. 5.2, Eq. 9), worked by hand on complex S, c and y, and the grid mean
    (1/n) 1^T x_hat.  A conjugated c, the wrong axis of the mean or a transposed
    product gives another number."""
    from types import SimpleNamespace
    S = np.array([[1 + 2j, 0], [3, -1j], [0, 2]])
    c = np.array([1, 2j, -1])
    prob = SimpleNamespace(qoi_kind="transpose", c=c, n=3)
    # c^T S = [1 (1+2j) + 2j 3 + (-1) 0, 1 0 + 2j (-1j) + (-1) 2] = [1 + 8j, 0]
    np.testing.assert_allclose(online.qoi_vector(prob, S), [1 + 8j, 0], rtol=0, atol=1e-15)
    # (1 + 8j)(2 - 1j) + 0 * 5 = 10 + 15j
    np.testing.assert_allclose(online.qoi(prob, S, np.array([[2 - 1j, 5]])), [10 + 15j], rtol=0, atol=1e-14)
    Sr = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 9.0]])
    mean = SimpleNamespace(qoi_kind="mean", c=None, n=3)
    np.testing.assert_allclose(online.qoi_vector(mean, Sr), [3.0, 5.0], rtol=0, atol=1e-15)
    # x_hat = S [1, -1] = [-1, -1, -4], mean -2
    np.testing.assert_allclose(online.qoi(mean, Sr, np.array([[1.0, -1.0]])), [-2.0], rtol=0, atol=1e-15)
