"""Device-side inputs of one context, kept alive next to it.

This is marshalling: it copies a problem's operator blocks (CSR), basis S,
right-hand side and QoI vector to device tensors, fills the C descriptor and
owns the context.  No arithmetic of the online stage happens here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def csr_to_device(A, device):
    A = A.tocsr()
    A.sort_indices()
    return (torch.from_numpy(A.indptr.astype(np.int64)).to(device),
            torch.from_numpy(A.indices.astype(np.int32)).to(device),
            torch.from_numpy(np.ascontiguousarray(A.data, dtype=np.float64)).to(device))


def basis_to_device(S, device, complex_valued=False):
    """n x r basis -> device tensor of shape (r, n) (column-major n x r, ldS = n)."""
    if isinstance(S, torch.Tensor):
        t = S.to(device)
        return t.T.contiguous()
    dt = np.complex128 if complex_valued else np.float64
    return torch.from_numpy(np.ascontiguousarray(np.asarray(S, dtype=dt).T)).to(device)


def theta_rule_code(rule):
    """C-ABI code of a problem's theta rule."""
    return {"linear": api.SAS_THETA_LINEAR, "pencil": api.SAS_THETA_PENCIL,
            "delay": api.SAS_THETA_DELAY}[rule]


class AffineSolver:
    """Context for A(p) = sum_k theta_k(p) A_k built from a workload problem."""

    def __init__(self, prob, S, J, mode=api.SAS_MODE_PLAIN, device="cuda", S_device=None,
                 blocks_device=None, b_device=None, c_device=None, weights=None):
        self.prob = prob
        self.device = device
        cplx = bool(prob.complex_valued)
        self.complex_valued = cplx
        self.blocks = blocks_device or [csr_to_device(A, device) for A in prob.blocks]
        self.S = S_device if S_device is not None else basis_to_device(S, device, cplx)
        bdt = np.complex128 if cplx else np.float64
        self.b = b_device if b_device is not None else \
            torch.from_numpy(np.ascontiguousarray(prob.b, dtype=bdt)).to(device)
        qk = api.SAS_QOI_NONE
        self.c = None
        if getattr(prob, "qoi_kind", None) == "mean":
            qk = api.SAS_QOI_MEAN
        elif getattr(prob, "qoi_kind", None) == "transpose":
            qk = api.SAS_QOI_TRANSPOSE
            self.c = c_device if c_device is not None else \
                torch.from_numpy(np.ascontiguousarray(prob.c, dtype=np.float64)).to(device)
        rule = theta_rule_code(prob.theta_rule)
        self.J = np.asarray(J, dtype=np.int64)
        self.desc = api._affine_desc(prob.n, prob.r, len(self.J), self.blocks, self.S, self.J,
                                     self.b, rule, mode, qk, self.c, cplx, weights)
        self.mode = mode
        self.r = prob.r
        self.s = len(self.J)
        self.n = prob.n
        self.ctx = api.subapsnap_setup_affine(self.desc)

    def close(self):
        if self.ctx is not None:
            api.subapsnap_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- marshalled calls
    def solve(self, params, out_kind, out, flags=None, rho=None, stream=None):
        api.subapsnap_solve_batch(self.ctx, params, params.shape[0], out_kind, out, flags, rho, stream)

    def residual(self, params, Y, rho, stream=None):
        api.subapsnap_residual(self.ctx, params, params.shape[0], Y, rho, stream)

    def reconstruct(self, Y, out, stream=None):
        api.subapsnap_reconstruct(self.ctx, Y, Y.shape[0], out, stream)

    def true_residual(self, params, X, rho, stream=None):
        api.subapsnap_true_residual(self.ctx, params, params.shape[0], X, rho, stream)


def poisson_precond(prob, params):
    """Fast Poisson preconditioner for the grid workloads: M = alpha L + beta I per column.

    2-D diffusion, A(p) = A_0 + sum p_k A_k with A_0 = h^-2 L: alpha = h^-2, beta = 0.
    Transfer function, A = i omega E - A_0 with A_0 = -h^-2 L: alpha = h^-2,
    beta = i omega mean(E).  Returns None for the other workloads."""
    P = np.atleast_2d(np.asarray(params, dtype=np.float64))
    grid = tuple(getattr(prob, "grid", ()) or ())
    if prob.name in ("diffusion_2d", "surrogate_diffusion_2d") and len(grid) == 2:
        h = 1.0 / (grid[0] + 1)
        coef = np.zeros((P.shape[0], 4))
        coef[:, 0] = 1.0 / (h * h)
        return {"dims": grid, "coef": coef}
    if prob.name == "transfer_function" and len(grid) == 3:
        h = 1.0 / (grid[0] + 1)
        ebar = float(prob.blocks[1].diagonal().mean())
        coef = np.zeros((P.shape[0], 4))
        coef[:, 0] = 1.0 / (h * h)
        coef[:, 3] = P[:, 0] * ebar
        return {"dims": grid, "coef": coef}
    return None


def snapshot_solve(prob, params, X, blocks_device=None, b_device=None, warm=False, tol=1e-12,
                   maxit=20000, device="cuda", allow_noconv=False, mixed=False, precond=None, method="cg"):
    """Batched Krylov solves A(p_j) x_j = b on the device into X (B, n); (iterations, true residuals)."""
    cplx = bool(prob.complex_valued)
    blocks = blocks_device or [csr_to_device(A, device) for A in prob.blocks]
    bdt = np.complex128 if cplx else np.float64
    b = b_device if b_device is not None else \
        torch.from_numpy(np.ascontiguousarray(prob.b, dtype=bdt)).to(device)
    P = np.atleast_2d(np.asarray(params, dtype=np.float64))
    desc = api._affine_desc(prob.n, P.shape[0], P.shape[0], blocks, None, None, b,
                            theta_rule_code(prob.theta_rule), api.SAS_MODE_PLAIN, api.SAS_QOI_NONE,
                            None, cplx)
    return api.subapsnap_krylov_affine(desc, P, X, warm=warm, tol=tol, maxit=maxit,
                                       allow_noconv=allow_noconv, mixed=mixed, precond=precond, method=method)


def snapshot_basis(prob, blocks_device=None, b_device=None, params=None, tol=1e-12, maxit=20000,
                   device="cuda", mixed=False, precond=None):
    """Offline stage on the device (Alg. 1 steps 1-2): snapshot solves, then TSQR.

    Returns (S, info): S is the (r, n) device tensor of the orthonormal basis
    (the column-major n x r matrix the online contexts take); info holds the
    iteration counts, the true residuals of the solves and R."""
    cplx = bool(prob.complex_valued)
    P = prob.snap_params if params is None else params
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    X = torch.empty((P.shape[0], prob.n), dtype=torch.complex128 if cplx else torch.float64, device=device)
    it, rel = snapshot_solve(prob, P, X, blocks_device, b_device, tol=tol, maxit=maxit, device=device,
                             mixed=mixed, precond=precond)
    R = api.subapsnap_tsqr(X)
    return X, {"iters": it, "relres": rel, "R": R}


def select_rows(prob, S_device, blocks_device, p_sel, s, device="cuda"):
    """CPQR-in-rounds row selection on the device; returns (J, gaps) on the host."""
    cplx = bool(prob.complex_valued)
    rule = theta_rule_code(prob.theta_rule)
    desc = api._affine_desc(prob.n, prob.r, s, blocks_device, S_device, None, None, rule,
                            api.SAS_MODE_PLAIN, api.SAS_QOI_NONE, None, cplx)
    return api.subapsnap_select_rows_affine(desc, p_sel, s)


def leverage_rows(prob, S_device, blocks_device, p_sel, s, u, device="cuda"):
    """Leverage-score sampling on the device scores of [A(p_sel) S, b]: (J, w, scores)."""
    cplx = bool(prob.complex_valued)
    bdt = np.complex128 if cplx else np.float64
    b = torch.from_numpy(np.ascontiguousarray(prob.b, dtype=bdt)).to(device)
    desc = api._affine_desc(prob.n, prob.r, s, blocks_device, S_device, None, b,
                            theta_rule_code(prob.theta_rule), api.SAS_MODE_PLAIN, api.SAS_QOI_NONE,
                            None, cplx)
    scores = api.subapsnap_leverage_scores_affine(desc, p_sel)
    J, w = api.subapsnap_sample_rows_leverage(scores, s, u)
    return J, w, scores


def select_rows_union(prob, S_device, blocks_device, points, s_each):
    """Union of the device CPQR picks at each row of ``points`` (first appearance order)."""
    cplx = bool(prob.complex_valued)
    desc = api._affine_desc(prob.n, prob.r, s_each, blocks_device, S_device, None, None,
                            theta_rule_code(prob.theta_rule), api.SAS_MODE_PLAIN, api.SAS_QOI_NONE,
                            None, cplx)
    return api.subapsnap_select_rows_union_affine(desc, points, s_each)


class NearestPointSolver:
    """Row set chosen per parameter: the CPQR rows of its nearest selection point.

    One AffineSolver per point shares the device basis, blocks, b and c; a
    batch is split by ``subapsnap_nearest_points`` and each group is solved
    by its point's context, the results scattered back in input order.
    """

    def __init__(self, prob, S, points, s, mode=api.SAS_MODE_PLAIN, device="cuda", S_device=None,
                 blocks_device=None):
        cplx = bool(prob.complex_valued)
        self.blocks = blocks_device or [csr_to_device(A, device) for A in prob.blocks]
        self.S = S_device if S_device is not None else basis_to_device(S, device, cplx)
        self.points = np.ascontiguousarray(np.atleast_2d(np.asarray(points, dtype=np.float64)))
        self.J = [select_rows(prob, self.S, self.blocks, pt, s)[0] for pt in self.points]
        bdt = np.complex128 if cplx else np.float64
        b = torch.from_numpy(np.ascontiguousarray(prob.b, dtype=bdt)).to(device)
        c = None if getattr(prob, "c", None) is None else \
            torch.from_numpy(np.ascontiguousarray(prob.c, dtype=np.float64)).to(device)
        self.solvers = [AffineSolver(prob, None, J, mode=mode, device=device, S_device=self.S,
                                     blocks_device=self.blocks, b_device=b, c_device=c) for J in self.J]

    def close(self):
        for sv in self.solvers:
            sv.close()

    def reconstruct(self, Y, out, stream=None):
        """x_hat = S y: every point's context holds the same basis."""
        self.solvers[0].reconstruct(Y, out, stream)

    def assign(self, params):
        P = params.detach().cpu().numpy() if hasattr(params, "detach") else np.asarray(params)
        return api.subapsnap_nearest_points(P, self.points)

    def solve(self, params, out_kind, out, flags=None, rho=None, stream=None):
        if stream is not None:
            with torch.cuda.stream(stream):
                return self.solve(params, out_kind, out, flags, rho, None)
        idx = self.assign(params)
        if np.all(np.diff(idx) >= 0):
            # parameters already grouped by point: every group is a contiguous slice
            bounds = np.searchsorted(idx, np.arange(len(self.solvers) + 1))
            for i, sv in enumerate(self.solvers):
                lo, hi = int(bounds[i]), int(bounds[i + 1])
                if hi > lo:
                    sv.solve(params[lo:hi], out_kind, out[lo:hi], None if flags is None else flags[lo:hi],
                             None if rho is None else rho[lo:hi], stream)
            return idx
        for i, sv in enumerate(self.solvers):
            sel = np.nonzero(idx == i)[0]
            if sel.size == 0:
                continue
            g = torch.from_numpy(sel).to(params.device)
            Pg = params.index_select(0, g).contiguous()
            og = out.new_empty((sel.size,) + tuple(out.shape[1:]))
            fg = None if flags is None else flags.new_zeros(sel.size)
            rg = None if rho is None else rho.new_empty(sel.size)
            sv.solve(Pg, out_kind, og, fg, rg, stream)
            out.index_copy_(0, g, og)
            if flags is not None:
                flags.index_copy_(0, g, fg)
            if rho is not None:
                rho.index_copy_(0, g, rg)
        return idx


class KernelSolver:
    """Context for A(sigma, lambda) = K_sigma + lambda I on points X (Gaussian kernel)."""

    def __init__(self, prob, S, J, mode=api.SAS_MODE_PLAIN, device="cuda", S_device=None,
                 X_device=None, b_device=None):
        self.prob = prob
        self.X = X_device if X_device is not None else \
            torch.from_numpy(np.ascontiguousarray(prob.X, dtype=np.float64)).to(device)
        self.S = S_device if S_device is not None else basis_to_device(S, device)
        self.b = b_device if b_device is not None else \
            torch.from_numpy(np.ascontiguousarray(prob.b, dtype=np.float64)).to(device)
        self.J = np.asarray(J, dtype=np.int64)
        self.desc = api._kernel_desc(prob.n, prob.X.shape[1], prob.r, len(self.J), self.X, self.S,
                                     self.J, self.b, mode)
        self.r, self.s, self.n, self.mode = prob.r, len(self.J), prob.n, mode
        self.ctx = api.subapsnap_setup_kernel(self.desc)

    def close(self):
        if self.ctx is not None:
            api.subapsnap_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, params, out_kind, out, flags=None, rho=None, stream=None):
        api.subapsnap_solve_batch(self.ctx, params, params.shape[0], out_kind, out, flags, rho, stream)

    def residual(self, params, Y, rho, stream=None):
        api.subapsnap_residual(self.ctx, params, params.shape[0], Y, rho, stream)


def point_shard(n, rank, world):
    """Contiguous block of the n points that rank owns (blocks differ by at most one)."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return slice(lo, lo + base + (1 if rank < extra else 0))


def allreduce_rows(M, dist_mod):
    """Sum the shards' partial kernel rows in place: the one exchange of the point split."""
    if dist_mod is not None and dist_mod.get_world_size() > 1:
        dist_mod.all_reduce(M, op=dist_mod.ReduceOp.SUM)
    return M


class KernelShard:
    """One shard of the points of a Gaussian-kernel problem: its context forms the partial rows
    M_g = K_sigma(X_J, X_g) S_g (+ lambda S_J on the shard that owns it); the sum over the shards
    is the full M, which any shard's context then solves."""

    def __init__(self, X, S, XJ, SJ, bJ, shard, r, s, mode=api.SAS_MODE_PLAIN, owns_lambda=False):
        n_all = X.shape[0]
        self.X = X[shard].contiguous()
        self.S = S  # (r, N) row-major: the shard's rows start at shard.start with ldS = N
        self.SJ = SJ if owns_lambda else torch.zeros_like(SJ)
        self.XJ, self.bJ = XJ, bJ
        ng = shard.stop - shard.start
        base = api.KernelDesc()
        base.n, base.d, base.r, base.s, base.mode = int(ng), int(X.shape[1]), int(r), int(s), mode
        base.X = api._ptr(self.X)
        base.S = S.data_ptr() + 8 * shard.start
        base.ldS = int(n_all)
        base.J = None
        base.b = None
        self.desc = api.KernelShardDesc(base=base, XJ=api._ptr(self.XJ), SJ=api._ptr(self.SJ),
                                        bJ=api._ptr(self.bJ))
        self.r, self.s = r, s
        self.ctx = api.subapsnap_setup_kernel_shard(self.desc)

    @classmethod
    def from_full(cls, X, S, b, J, rank, world, r, mode=api.SAS_MODE_PLAIN):
        Jd = torch.as_tensor(np.asarray(J, dtype=np.int64), device=X.device)
        XJ = X.index_select(0, Jd).contiguous()
        SJ = S.index_select(1, Jd).contiguous()  # (r, s): column-major s x r with ld s
        bJ = b.index_select(0, Jd).contiguous()
        return cls(X, S, XJ, SJ, bJ, point_shard(X.shape[0], rank, world), r, len(J), mode,
                   owns_lambda=rank == 0)

    def rows(self, params, M, stream=None):
        api.subapsnap_kernel_rows(self.ctx, params, params.shape[0], M, stream)

    def solve_rows(self, params, M, Y, flags=None, rho=None, stream=None):
        api.subapsnap_solve_batch_rows(self.ctx, params, params.shape[0], M, Y, flags, rho, stream)

    def close(self):
        if self.ctx is not None:
            api.subapsnap_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def select_rows_kernel(prob, X_device, S_device, p_sel, s):
    """CPQR-in-rounds row selection for the Gaussian-kernel family; (J, gaps) on the host."""
    J0 = np.arange(s, dtype=np.int64)
    b = torch.zeros(1, dtype=torch.float64, device=X_device.device)
    desc = api._kernel_desc(prob.n, prob.X.shape[1], prob.r, s, X_device, S_device, J0, b,
                            api.SAS_MODE_PLAIN)
    return api.subapsnap_select_rows_kernel(desc, p_sel, s)
