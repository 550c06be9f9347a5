"""GPU parity of the offline stage (Alg. 1 steps 1-2) against the oracle, through the C-ABI.

Tolerances
  Snapshot solves: the batched COCG stops at ||b - A x|| / ||b|| <= tol; the
    true residual recomputed by the oracle's own matrix must be <= 10 tol (the
    updated and the true residual drift apart by ~kappa(A) u), and the distance
    to the oracle's direct solve is bounded by kappa(A) times the residual.
  TSQR: with diag(R) >= 0 the thin QR of a full-rank X is unique, so Q and R
    are compared with the oracle's entry by entry: |Q - Q_o| <= 1e-12 and
    |R - R_o| <= 1e-12 |R| for well-conditioned X (the perturbation of the QR
    factors is ~kappa(X) u).  For numerically rank-deficient X only what is
    unique is compared: Q^H Q = I, X = Q R and |R| against the oracle's on the
    well-determined leading columns.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect with -m "not gpu"
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import online, problem as oproblem, selection, snapshots  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import (AffineSolver, csr_to_device, select_rows,  # noqa: E402
                                           snapshot_basis, snapshot_solve)
from workloads import get_config  # noqa: E402

DEV = "cuda"

SMALL = [("reaction_diffusion_1d", dict(n=1000, r=8, s=16, m=20)),
         ("diffusion_2d", dict(N=48, r=60, s=120, m=40)),
         ("transfer_function", dict(N=9, r=20, s=50, m=40)),
         ("delay_system", dict(n=3000, r=16, s=32, m=40))]


def _tensor(a, cplx):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128 if cplx else np.float64)).to(DEV)


@pytest.mark.parametrize("mixed", [False, True], ids=["plain", "mixed"])
@pytest.mark.parametrize("name,kw", SMALL, ids=[c[0] for c in SMALL])
def test_snapshot_solves_match_direct_solves(name, kw, mixed):
    prob = get_config(name, **kw)
    cplx = prob.complex_valued
    P = prob.snap_params
    X = torch.empty((len(P), prob.n), dtype=torch.complex128 if cplx else torch.float64, device=DEV)
    tol = 1e-10
    it, rel = snapshot_solve(prob, P, X, tol=tol, maxit=50000, mixed=mixed)
    Xg = X.cpu().numpy()
    worst_err = 0.0
    for j, p in enumerate(P):
        A = oproblem.full_matrix(prob, p)
        xo = snapshots.solve_full(prob, p)
        res = np.linalg.norm(A @ Xg[j] - prob.b) / np.linalg.norm(prob.b)
        # convergence is declared on the float64 true residual
        assert rel[j] <= tol and res <= 2 * tol, (j, res, rel[j])
        err = np.linalg.norm(Xg[j] - xo) / np.linalg.norm(xo)
        worst_err = max(worst_err, err)
        # forward error <= kappa(A) * residual (kappa from a dense SVD at these sizes)
        if prob.n <= 2500:
            sv = np.linalg.svd(A.toarray(), compute_uv=False)
            assert err <= sv[0] / sv[-1] * 10 * tol, (j, err)
    print(f"{name} {'mixed' if mixed else 'plain'}: iterations {it.min()}..{it.max()}, max true residual {rel.max():.2e}, "
          f"max error vs direct {worst_err:.2e}")


def test_warm_start_from_subapsnap_output():
    """x_hat from the online stage as the start vector (Sec. 3.2): fewer iterations, same bar."""
    prob = get_config("diffusion_2d", N=48, r=20, s=40, m=8)
    S = snapshots.orthonormal_basis(snapshots.snapshot_matrix(prob))
    V = np.asarray(oproblem.full_matrix(prob, prob.sel_param) @ S)
    J, _ = selection.cpqr_rows(V, prob.s)
    params = prob.test_params[:8]
    Y, _ = online.solve_many(prob, S, J, params)
    Xhat = Y @ S.T
    tol = 1e-11
    Xw = _tensor(Xhat, False)
    it_w, rel_w = snapshot_solve(prob, params, Xw, warm=True, tol=tol)
    Xc = torch.empty_like(Xw)
    it_c, rel_c = snapshot_solve(prob, params, Xc, warm=False, tol=tol)
    assert (rel_w <= tol).all() and (rel_c <= tol).all()
    Xm = _tensor(Xhat, False)
    it_m, rel_m = snapshot_solve(prob, params, Xm, warm=True, tol=tol, mixed=True)
    assert (rel_m <= tol).all()
    assert (it_w < it_c).all(), (it_w, it_c)
    print(f"warm start: {it_w.mean():.0f} iterations against {it_c.mean():.0f} from zero "
          f"({it_m.mean():.0f} with float32 iterates)")


def test_krylov_iteration_limit_and_bad_arguments():
    prob = get_config("diffusion_2d", N=32, r=4, s=8, m=4)
    X = torch.empty((4, prob.n), dtype=torch.float64, device=DEV)
    with pytest.raises(api.SasError) as ei:
        snapshot_solve(prob, prob.snap_params, X, tol=1e-14, maxit=3)
    assert ei.value.code == api.SAS_ENOCONV
    it, rel = snapshot_solve(prob, prob.snap_params, X, tol=1e-14, maxit=3, allow_noconv=True)
    assert (it == 3).all() and np.isfinite(rel).all()
    with pytest.raises(api.SasError):
        snapshot_solve(prob, prob.snap_params, X, tol=-1.0)


@pytest.mark.parametrize("n,r,cplx", [(5000, 37, False), (100_000, 60, False), (5000, 20, True),
                                      (2000, 80, True), (777, 1, False), (130, 64, False)])
def test_tsqr_matches_oracle_on_full_rank(n, r, cplx):
    rng = np.random.default_rng(n + r)
    Xh = rng.standard_normal((n, r))
    if cplx:
        Xh = Xh + 1j * rng.standard_normal((n, r))
    Xh[:, 0] *= 1e3  # uneven column scales, still well conditioned
    X = _tensor(Xh.T, cplx)
    Q = torch.empty_like(X)
    R = api.subapsnap_tsqr(X, Q)
    Qo, Ro = snapshots.thin_qr(Xh)
    Qg = Q.cpu().numpy().T
    np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12)
    np.testing.assert_allclose(R, Ro, rtol=0, atol=1e-12 * np.abs(Ro).max())
    # in place
    api.subapsnap_tsqr(X)
    np.testing.assert_array_equal(X.cpu().numpy().T, Qg)


@pytest.mark.parametrize("name,kw", SMALL[:1] + SMALL[2:], ids=[c[0] for c in SMALL[:1] + SMALL[2:]])
def test_tsqr_on_rank_deficient_snapshots(name, kw):
    """Snapshot matrices with kappa ~ 1e15 .. 1e22: what is unique about their QR."""
    prob = get_config(name, **kw)
    Xh = snapshots.snapshot_matrix(prob)
    cplx = prob.complex_valued
    X = _tensor(Xh.T, cplx)
    R = api.subapsnap_tsqr(X, X)
    Q = X.cpu().numpy().T
    r = Xh.shape[1]
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(Q @ R, Xh, atol=1e-14 * np.linalg.norm(Xh, 2))
    assert np.allclose(np.tril(R, -1), 0)
    d = np.diag(R)
    assert (d.real >= 0).all() and (d.imag == 0).all()
    _, Ro = snapshots.thin_qr(Xh)
    lead = np.abs(np.diag(Ro)) > 1e-8 * np.abs(Ro[0, 0])
    k = int(np.argmin(lead)) if not lead.all() else r
    np.testing.assert_allclose(np.abs(np.diag(R))[:k], np.abs(np.diag(Ro))[:k], rtol=1e-6)


def test_offline_then_online_pipeline():
    """Snapshots, basis and rows all on the device, then the online stage; the result
    has the same quality as the oracle's pipeline (x_hat true residual)."""
    prob = get_config("diffusion_2d", N=48, r=30, s=60, m=40)
    blocks = [csr_to_device(A, DEV) for A in prob.blocks]
    S, info = snapshot_basis(prob, blocks_device=blocks, tol=1e-12, mixed=True)
    assert (info["relres"] <= 1e-12).all()
    J, _ = select_rows(prob, S, blocks, prob.sel_param, prob.s)
    So = snapshots.orthonormal_basis(snapshots.snapshot_matrix(prob))
    Vo = np.asarray(oproblem.full_matrix(prob, prob.sel_param) @ So)
    Jo, _ = selection.cpqr_rows(Vo, prob.s)
    overlap = len(set(J.tolist()) & set(Jo.tolist())) / prob.s
    sv = AffineSolver(prob, None, J, mode=api.SAS_MODE_PLAIN, device=DEV, S_device=S, blocks_device=blocks)
    params = prob.test_params
    Pd = torch.from_numpy(np.ascontiguousarray(params)).to(DEV)
    Xg = torch.empty((len(params), prob.n), dtype=torch.float64, device=DEV)
    sv.solve(Pd, api.SAS_OUT_XHAT, Xg)
    Xg = Xg.cpu().numpy()
    sv.close()
    Yo, _ = online.solve_many(prob, So, Jo, params)
    Xo = Yo @ So.T
    res_g, res_o = [], []
    for j, p in enumerate(params):
        A = oproblem.full_matrix(prob, p)
        nb = np.linalg.norm(prob.b)
        res_g.append(np.linalg.norm(A @ Xg[j] - prob.b) / nb)
        res_o.append(np.linalg.norm(A @ Xo[j] - prob.b) / nb)
    res_g, res_o = np.array(res_g), np.array(res_o)
    assert (res_g <= 10 * res_o + 1e-9).all(), (res_g.max(), res_o.max())
    print(f"pipeline: x_hat residual max {res_g.max():.2e} (oracle pipeline {res_o.max():.2e}), "
          f"rows shared with the oracle's J {overlap:.0%}")


def test_dense_rows_take_the_unstaged_path():
    """Eight blocks of 9-point stencils: ~70 stored entries per row, more than a tile's
    shared-memory stage holds, so the product reads the CSR arrays from global memory."""
    import types
    import scipy.sparse as sp
    N = 40
    n = N * N
    rng = np.random.default_rng(11)
    one = np.ones(N)
    T1 = sp.diags([-one[1:], 2 * one, -one[1:]], [-1, 0, 1])
    I = sp.identity(N)
    lap = (sp.kron(I, T1) + sp.kron(T1, I)).tocsr()
    blocks = [lap + sp.identity(n) * 0.1]
    for k in range(7):  # SPD 9-point blocks with random positive weights
        w = rng.uniform(0.5, 1.5, n)
        W = sp.diags(w)
        Tp = sp.diags([one[1:], 2 * one, one[1:]], [-1, 0, 1])  # positive semidefinite
        M = sp.kron(Tp, Tp)
        blocks.append((W @ M @ W * 0.05 + sp.identity(n) * 2.0).tocsr())
    prob = types.SimpleNamespace(name="dense_rows", n=n, blocks=blocks, theta_rule="linear",
                                 b=rng.standard_normal(n), complex_valued=False)
    per_row = sum(B.nnz for B in blocks) / n
    assert per_row * 128 > 4096, per_row
    P = rng.uniform(0.0, 1.0, (5, 7))
    for mixed in (False, True):
        X = torch.empty((5, n), dtype=torch.float64, device=DEV)
        it, rel = snapshot_solve(prob, P, X, tol=1e-10, mixed=mixed)
        Xg = X.cpu().numpy()
        for j, p in enumerate(P):
            xo = snapshots.solve_full(prob, p)
            A = oproblem.full_matrix(prob, p)
            assert np.linalg.norm(A @ Xg[j] - prob.b) / np.linalg.norm(prob.b) <= 2e-10
            assert np.linalg.norm(Xg[j] - xo) / np.linalg.norm(xo) <= 1e-7
        print(f"unstaged rows ({per_row:.0f} per row), {'mixed' if mixed else 'plain'}: iterations {it.max()}")


def test_batch_limits_and_single_column():
    prob = get_config("diffusion_2d", N=20, r=3, s=6, m=4)
    X = torch.empty((1, prob.n), dtype=torch.float64, device=DEV)
    it, rel = snapshot_solve(prob, prob.snap_params[:1], X, tol=1e-12)
    xo = snapshots.solve_full(prob, prob.snap_params[0])
    assert np.linalg.norm(X.cpu().numpy()[0] - xo) / np.linalg.norm(xo) <= 1e-9
    with pytest.raises(api.SasError):
        Xb = torch.empty((257, prob.n), dtype=torch.float64, device=DEV)
        snapshot_solve(prob, np.tile(prob.snap_params[:1], (257, 1)), Xb)


@pytest.mark.parametrize("mixed", [False, True], ids=["plain", "mixed"])
@pytest.mark.parametrize("name,kw", [("diffusion_2d", dict(N=48, r=20, s=40, m=4)),
                                     ("transfer_function", dict(N=9, r=20, s=50, m=4))],
                         ids=["diffusion_2d", "transfer_function"])
def test_poisson_preconditioner(name, kw, mixed):
    """Fast Poisson preconditioner (DST along each axis): same answers as the direct
    solves, in far fewer iterations than the diagonal preconditioner."""
    from paper_2510_04825_gb300.solver import poisson_precond
    prob = get_config(name, **kw)
    cplx = prob.complex_valued
    P = prob.snap_params
    dt = torch.complex128 if cplx else torch.float64
    tol = 1e-10
    Xp = torch.empty((len(P), prob.n), dtype=dt, device=DEV)
    it_p, rel_p = snapshot_solve(prob, P, Xp, tol=tol, mixed=mixed, precond=poisson_precond(prob, P))
    Xj = torch.empty_like(Xp)
    it_j, _ = snapshot_solve(prob, P, Xj, tol=tol, mixed=mixed)
    assert (rel_p <= tol).all()
    Xg = Xp.cpu().numpy()
    for j, p in enumerate(P):
        xo = snapshots.solve_full(prob, p)
        A = oproblem.full_matrix(prob, p)
        assert np.linalg.norm(A @ Xg[j] - prob.b) / np.linalg.norm(prob.b) <= 2 * tol
        assert np.linalg.norm(Xg[j] - xo) / np.linalg.norm(xo) <= 1e-7
    assert it_p.max() < it_j.max(), (it_p.max(), it_j.max())
    print(f"{name} {'mixed' if mixed else 'plain'}: Poisson-preconditioned iterations {it_p.min()}..{it_p.max()}, "
          f"diagonal {it_j.min()}..{it_j.max()}")


def test_poisson_preconditioner_arguments():
    from paper_2510_04825_gb300.solver import poisson_precond
    prob = get_config("diffusion_2d", N=20, r=3, s=6, m=4)
    X = torch.empty((3, prob.n), dtype=torch.float64, device=DEV)
    pc = poisson_precond(prob, prob.snap_params)
    bad = dict(pc, dims=(20, 21))
    with pytest.raises(api.SasError):
        snapshot_solve(prob, prob.snap_params, X, precond=bad)
    cplx = dict(pc, coef=pc["coef"] + np.array([0, 1.0, 0, 0]))
    with pytest.raises(api.SasError):
        snapshot_solve(prob, prob.snap_params, X, precond=cplx)


def _convection_diffusion(N, cplx):
    """Nonsymmetric family: 2-D convection-diffusion (upwind convection), A(p) = A_0 + p A_1
    with A_1 a positive reaction term; complex version: the pencil i omega E - A_0 on the
    same nonsymmetric A_0 (negated)."""
    import types
    import scipy.sparse as sp
    rng = np.random.default_rng(21)
    n = N * N
    h = 1.0 / (N + 1)
    one = np.ones(N)
    T1 = sp.diags([-one[1:], 2 * one, -one[1:]], [-1, 0, 1])
    Dx = sp.diags([-one[1:], one], [-1, 0])  # upwind first difference
    I = sp.identity(N)
    L = (sp.kron(I, T1) + sp.kron(T1, I)) / h ** 2
    C = 40.0 * (sp.kron(I, Dx) + 0.5 * sp.kron(Dx, I)) / h
    A0 = (L + C).tocsr()
    b = rng.standard_normal(n)
    if not cplx:
        A1 = sp.diags(rng.uniform(0.5, 1.5, n)).tocsr()
        return types.SimpleNamespace(name="convection_diffusion", n=n, blocks=[A0, A1], theta_rule="linear",
                                     b=b, complex_valued=False), rng.uniform(0.0, 10.0, (6, 1))
    E = sp.diags(rng.uniform(0.5, 1.5, n)).tocsr()
    return types.SimpleNamespace(name="convection_diffusion_pencil", n=n, blocks=[(-A0).tocsr(), E],
                                 theta_rule="pencil", b=b.astype(np.complex128), complex_valued=True), \
        np.logspace(0, 3, 6)[:, None]


@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex"])
def test_bicgstab_on_a_nonsymmetric_family(cplx):
    prob, P = _convection_diffusion(30, cplx)
    dt = torch.complex128 if cplx else torch.float64
    X = torch.empty((len(P), prob.n), dtype=dt, device=DEV)
    tol = 1e-10
    it, rel = snapshot_solve(prob, P, X, tol=tol, maxit=5000, method="bicgstab")
    assert (rel <= tol).all()
    Xg = X.cpu().numpy()
    for j, p in enumerate(P):
        xo = snapshots.solve_full(prob, p)
        A = oproblem.full_matrix(prob, p)
        assert np.linalg.norm(A @ Xg[j] - prob.b) / np.linalg.norm(prob.b) <= 2 * tol
        assert np.linalg.norm(Xg[j] - xo) / np.linalg.norm(xo) <= 1e-6
    # warm start from the solution's neighbourhood takes fewer iterations
    Xw = torch.from_numpy(np.ascontiguousarray(Xg * (1 + 1e-6))).to(DEV)
    it_w, rel_w = snapshot_solve(prob, P, Xw, tol=tol, maxit=5000, method="bicgstab", warm=True)
    assert (rel_w <= tol).all() and (it_w < it).all()
    print(f"BiCGStab {'complex' if cplx else 'real'} nonsymmetric: iterations {it.min()}..{it.max()}, "
          f"warm {it_w.min()}..{it_w.max()}")


def test_bicgstab_on_a_symmetric_workload_and_arguments():
    prob = get_config("diffusion_2d", N=32, r=6, s=12, m=4)
    X = torch.empty((6, prob.n), dtype=torch.float64, device=DEV)
    it, rel = snapshot_solve(prob, prob.snap_params, X, tol=1e-10, maxit=5000, method="bicgstab")
    assert (rel <= 1e-10).all()
    for j, p in enumerate(prob.snap_params):
        xo = snapshots.solve_full(prob, p)
        assert np.linalg.norm(X.cpu().numpy()[j] - xo) / np.linalg.norm(xo) <= 1e-8
    with pytest.raises(api.SasError) as ei:
        snapshot_solve(prob, prob.snap_params, X, method="bicgstab", mixed=True)
    assert ei.value.code == api.SAS_ENOTSUP
