"""Snapshot bases S for the workloads (inputs of the online stage).

The online stage takes an orthonormal basis S of snapshot solutions
x(p_1), ..., x(p_r) as given.  This module produces it with generic solvers
that are neither the oracle nor the product library:
  * small and medium affine problems: sparse direct solves (scipy);
  * the 1-D tridiagonal problem: banded LU (scipy.linalg.solve_banded);
  * large 2-D diffusion problems: preconditioned CG on the GPU with torch,
    preconditioned by the constant-coefficient Laplacian, inverted with a
    sine transform (see ``diffusion_pcg``);
followed by a thin QR (numpy / torch) that orthonormalises the columns.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _A(prob, p):
    p = np.atleast_1d(np.asarray(p, dtype=np.float64))
    if prob.theta_rule == "linear":
        A = prob.blocks[0].copy()
        for k in range(1, len(prob.blocks)):
            A = A + p[k - 1] * prob.blocks[k]
        return A.tocsc()
    if prob.theta_rule == "pencil":
        return (1j * p[0] * prob.blocks[1] - prob.blocks[0]).tocsc()
    if prob.theta_rule == "delay":
        return (1j * p[0] * prob.blocks[0] - prob.blocks[1]
                - np.exp(1j * p[0] * p[1]) * prob.blocks[2]).tocsc()
    raise ValueError(prob.theta_rule)


def _tridiagonal_solve(A, b):
    """A tridiagonal sparse matrix: banded LU (LAPACK gbsv through scipy)."""
    A = A.tocsr()
    n = A.shape[0]
    ab = np.zeros((3, n), dtype=np.result_type(A.dtype, b.dtype))
    ab[0, 1:] = A.diagonal(1)
    ab[1] = A.diagonal(0)
    ab[2, :-1] = A.diagonal(-1)
    return sla.solve_banded((1, 1), ab, b)


def snapshot_solutions(prob) -> np.ndarray:
    """X = [x(p_1), ..., x(p_r)] (n x r) by direct solves."""
    if prob.name == "reaction_diffusion_1d":
        d = prob.meta["d"]
        cols = []
        for p in prob.snap_params[:, 0]:
            ab = np.zeros((3, prob.n))
            ab[0, 1:] = -1.0
            ab[1] = 2.0 + p * d
            ab[2, :-1] = -1.0
            cols.append(sla.solve_banded((1, 1), ab, prob.b))
        return np.stack(cols, 1)
    if hasattr(prob, "X"):  # kernel ridge, small N: dense solves
        from .operators import gaussian_kernel_block
        cols = []
        for sig, lam in prob.snap_params:
            K = gaussian_kernel_block(prob.X, prob.X, sig) + lam * np.eye(prob.n)
            cols.append(np.linalg.solve(K, prob.b))
        return np.stack(cols, 1)
    if prob.theta_rule == "delay":  # tridiagonal at every parameter
        return np.stack([_tridiagonal_solve(_A(prob, p), prob.b) for p in prob.snap_params], 1)
    cols = [spla.spsolve(_A(prob, p), prob.b) for p in prob.snap_params]
    return np.stack(cols, 1)


def delay_basis_torch(prob, device="cuda"):
    """Orthonormal snapshot basis of the delay system on the device: banded LU solves
    on the host (n = 1e7 is a few seconds each), Gram-Schmidt on the device.
    Returns (S_rows (r, n) complex128, max relative residual of the solves)."""
    import torch
    X = snapshot_solutions(prob)
    res = []
    for k, p in enumerate(prob.snap_params):
        A = _A(prob, p)
        res.append(np.linalg.norm(A @ X[:, k] - prob.b) / np.linalg.norm(prob.b))
    Q = orthonormalise_torch(torch.from_numpy(X).to(device))
    return Q.T.contiguous(), float(np.max(res))


def orthonormalise(X: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(X, mode="reduced")
    return np.ascontiguousarray(Q)


def basis(prob) -> np.ndarray:
    """Orthonormal snapshot basis S (n x r) by direct solves."""
    return orthonormalise(snapshot_solutions(prob))


# ---------------------------------------------------------------------------
# Large 2-D diffusion problems: batched PCG on the GPU (torch).
# ---------------------------------------------------------------------------

def _dst1_last(v):
    """Unnormalised DST-I along the last axis: y_k = sum_j v_j sin(pi j k / (N+1))."""
    import torch
    N = v.shape[-1]
    z = torch.zeros(v.shape[:-1] + (2 * (N + 1),), dtype=v.dtype, device=v.device)
    z[..., 1:N + 1] = v
    z[..., N + 2:] = -torch.flip(v, dims=(-1,))
    Z = torch.fft.rfft(z, dim=-1)
    return -0.5 * Z[..., 1:N + 1].imag


def _dst2(u):
    return _dst1_last(_dst1_last(u).transpose(-1, -2)).transpose(-1, -2)


def diffusion_faces_torch(prob, params, device):
    """Face coefficients a = 1 + sum_k p_k psi_k for a batch of parameters.

    Returns (ax, ay) with ax[b, j, i_face] of shape (B, N, N+1) and
    ay[b, j_face, i] of shape (B, N+1, N), matching the CSR blocks of
    ``workloads.operators.diffusion_2d``.
    """
    import torch
    faces = prob.meta["faces"]
    P = torch.as_tensor(np.asarray(params, dtype=np.float64), device=device)
    N = prob.grid[0]
    ax = torch.ones((P.shape[0], N, N + 1), dtype=torch.float64, device=device)
    ay = torch.ones((P.shape[0], N + 1, N), dtype=torch.float64, device=device)
    for k, (fx, fy) in enumerate(faces):
        gx = torch.as_tensor(np.ascontiguousarray(fx.T), device=device)  # (N, N+1)
        gy = torch.as_tensor(np.ascontiguousarray(fy.T), device=device)  # (N+1, N)
        ax += P[:, k, None, None] * gx[None]
        ay += P[:, k, None, None] * gy[None]
    return ax, ay


def diffusion_apply_torch(u, ax, ay, h):
    """-div(a grad u) / h^2 on (B, N, N) arrays, u[b, j, i] = u_{i + N j}."""
    import torch.nn.functional as F
    up = F.pad(u, (1, 1, 1, 1))
    fx = ax * (up[:, 1:-1, 1:] - up[:, 1:-1, :-1])
    fy = ay * (up[:, 1:, 1:-1] - up[:, :-1, 1:-1])
    return -((fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :])) / (h * h)


def diffusion_pcg(prob, params, device="cuda", rtol=1e-11, maxit=400, group=None):
    """Solve A(p) x = b for a batch of parameters with Laplacian-preconditioned CG.

    The preconditioner is the constant-coefficient operator (a = 1), applied
    exactly through the 2-D sine transform; since 1 <= a(x; p) <= 1 + sum p_k,
    the preconditioned condition number is at most max a / min a.
    Returns a torch tensor X of shape (B, n) (float64, on ``device``) and the
    final relative residuals.
    """
    import torch
    N = prob.grid[0]
    h = 1.0 / (N + 1)
    params = np.atleast_2d(np.asarray(params, dtype=np.float64))
    B = params.shape[0]
    if group is None:
        group = max(1, min(B, int(2.0e9 // (N * N * 8 * 12))))
    k = torch.arange(1, N + 1, dtype=torch.float64, device=device)
    s2 = torch.sin(np.pi * k / (2 * (N + 1))) ** 2
    lam = (4.0 / (h * h)) * (s2[:, None] + s2[None, :])
    scale = (2.0 / (N + 1)) ** 2
    bvec = torch.as_tensor(np.asarray(prob.b, dtype=np.float64).reshape(N, N), device=device)
    out = torch.empty((B, N * N), dtype=torch.float64, device=device)
    finals = []
    for g0 in range(0, B, group):
        P = params[g0:g0 + group]
        ax, ay = diffusion_faces_torch(prob, P, device)
        b = bvec.expand(P.shape[0], N, N).clone()
        bn = torch.linalg.vector_norm(b.reshape(len(P), -1), dim=1)
        x = torch.zeros_like(b)
        r = b.clone()
        z = scale * _dst2(_dst2(r) / lam)
        p = z.clone()
        rz = (r * z).sum(dim=(1, 2))
        for _ in range(maxit):
            Ap = diffusion_apply_torch(p, ax, ay, h)
            alpha = rz / (p * Ap).sum(dim=(1, 2))
            x += alpha[:, None, None] * p
            r -= alpha[:, None, None] * Ap
            rel = torch.linalg.vector_norm(r.reshape(len(P), -1), dim=1) / bn
            if bool((rel < rtol).all()):
                break
            z = scale * _dst2(_dst2(r) / lam)
            rz_new = (r * z).sum(dim=(1, 2))
            p = z + (rz_new / rz)[:, None, None] * p
            rz = rz_new
        res = diffusion_apply_torch(x, ax, ay, h) - b
        finals.append((torch.linalg.vector_norm(res.reshape(len(P), -1), dim=1) / bn).cpu().numpy())
        out[g0:g0 + len(P)] = x.reshape(len(P), -1)
        del ax, ay, b, x, r, z, p
    return out, np.concatenate(finals)


def orthonormalise_torch(X):
    """Orthonormal basis of the columns of X (n x r) by Gram-Schmidt applied twice.

    Uses matrix products only (no LAPACK), so it runs in any process that has
    cuBLAS; the span equals that of a thin QR, up to column signs or phases.
    """
    import torch
    n, r = X.shape
    Q = torch.empty_like(X)
    for k in range(r):
        v = X[:, k].clone()
        for _ in range(2):
            if k:
                Qk = Q[:, :k]
                v = v - Qk @ (Qk.conj().T @ v)
        Q[:, k] = v / torch.linalg.vector_norm(v)
    return Q


def diffusion_basis_torch(prob, device="cuda", **kw):
    """Orthonormal snapshot basis of a 2-D diffusion workload on the device.

    Returns (S_rows, final_residuals) with S_rows of shape (r, n): row k is
    column k of S, i.e. the column-major n x r layout with leading dimension n.
    """
    import torch
    X, res = diffusion_pcg(prob, prob.snap_params, device=device, **kw)
    Q = orthonormalise_torch(X.T)
    return Q.T.contiguous(), res


# ---------------------------------------------------------------------------
# Transfer-function workload (i w E - A_0) x = b on an N^3 grid: batched
# preconditioned COCG on the GPU (torch).
# ---------------------------------------------------------------------------

def _dst1_axis_complex(v, axis):
    """Unnormalised DST-I of a complex tensor along ``axis``."""
    import torch
    v = v.movedim(axis, -1)
    N = v.shape[-1]
    z = torch.zeros(v.shape[:-1] + (2 * (N + 1),), dtype=v.dtype, device=v.device)
    z[..., 1:N + 1] = v
    z[..., N + 2:] = -torch.flip(v, dims=(-1,))
    y = 0.5j * torch.fft.fft(z, dim=-1)[..., 1:N + 1]
    return y.movedim(-1, axis)


def _dst3_complex(u):
    for ax in (-1, -2, -3):
        u = _dst1_axis_complex(u, ax)
    return u


def heat3d_apply_torch(u, h):
    """A_0 u = h^-2 (sum of 6 neighbours - 6 u) on (B, N, N, N), zero Dirichlet."""
    import torch.nn.functional as F
    up = F.pad(u, (1, 1, 1, 1, 1, 1)) if not u.is_complex() else \
        F.pad(u.real, (1, 1, 1, 1, 1, 1)) + 1j * F.pad(u.imag, (1, 1, 1, 1, 1, 1))
    s = (up[:, 2:, 1:-1, 1:-1] + up[:, :-2, 1:-1, 1:-1] + up[:, 1:-1, 2:, 1:-1]
         + up[:, 1:-1, :-2, 1:-1] + up[:, 1:-1, 1:-1, 2:] + up[:, 1:-1, 1:-1, :-2])
    return (s - 6.0 * u) / (h * h)


def transfer_cocg(prob, omegas, device="cuda", rtol=1e-11, maxit=300, group=None):
    """Solve (i w E - A_0) x = b for a batch of w by COCG.

    Preconditioner: (-A_0 + i w I)^{-1}, applied exactly with the 3-D sine
    transform.  With E = diag(e), e in [0.5, 1.5], the preconditioned matrix is
    I + i w (-A_0 + i w I)^{-1} (E - I), within 0.5 of the identity in norm.
    Both matrices are complex symmetric, so the conjugate-free CG (COCG)
    applies.  Returns (X (B, n) complex128 on device, final relative residuals).
    """
    import torch
    N = prob.grid[0]
    h = 1.0 / (N + 1)
    om = np.asarray(omegas, dtype=np.float64).reshape(-1)
    B = om.size
    if group is None:
        group = max(1, min(B, int(1.5e9 // (N ** 3 * 16 * 12))))
    k = torch.arange(1, N + 1, dtype=torch.float64, device=device)
    s2 = torch.sin(np.pi * k / (2 * (N + 1))) ** 2
    mu = (4.0 / (h * h)) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    scale = (2.0 / (N + 1)) ** 3
    e = torch.as_tensor(prob.meta["e"].reshape(N, N, N), device=device)
    bvec = torch.as_tensor(np.asarray(prob.b).reshape(N, N, N), device=device).to(torch.complex128)
    out = torch.empty((B, N ** 3), dtype=torch.complex128, device=device)
    finals = []
    for g0 in range(0, B, group):
        w = torch.as_tensor(om[g0:g0 + group], device=device)
        G = w.numel()
        iw = (1j * w)[:, None, None, None]
        pdiag = mu[None] + iw  # eigenvalues of -A_0 + i w I

        def A(v):
            return iw * e[None] * v - heat3d_apply_torch(v, h)

        def Pinv(v):
            return scale * _dst3_complex(_dst3_complex(v) / pdiag)

        b = bvec.expand(G, N, N, N).clone()
        bn = torch.linalg.vector_norm(b.reshape(G, -1), dim=1)
        x = torch.zeros_like(b)
        r = b.clone()
        z = Pinv(r)
        p = z.clone()
        rho = (r * z).sum(dim=(1, 2, 3))
        for _ in range(maxit):
            q = A(p)
            alpha = rho / (p * q).sum(dim=(1, 2, 3))
            x += alpha[:, None, None, None] * p
            r -= alpha[:, None, None, None] * q
            rel = torch.linalg.vector_norm(r.reshape(G, -1), dim=1) / bn
            if bool((rel < rtol).all()):
                break
            z = Pinv(r)
            rho_new = (r * z).sum(dim=(1, 2, 3))
            p = z + (rho_new / rho)[:, None, None, None] * p
            rho = rho_new
        res = A(x) - b
        finals.append((torch.linalg.vector_norm(res.reshape(G, -1), dim=1) / bn).cpu().numpy())
        out[g0:g0 + G] = x.reshape(G, -1)
    return out, np.concatenate(finals)


def transfer_basis_torch(prob, device="cuda", **kw):
    """Orthonormal snapshot basis of the transfer-function workload on the device.

    Returns (S_rows (r, n) complex128, final residuals); row k = column k of S.
    """
    import torch
    X, res = transfer_cocg(prob, prob.snap_params[:, 0], device=device, **kw)
    Q = orthonormalise_torch(X.T)
    return Q.T.contiguous(), res


# ---------------------------------------------------------------------------
# Kernel ridge regression: approximate snapshots (K_sigma + lambda I) x = y by
# a fixed number of CG iterations on the GPU (torch), the ten lambda values of
# one sigma sharing every kernel product.
# ---------------------------------------------------------------------------

def kernel_ridge_cr(prob, X, sigma, lams, iters=40, block=8192):
    """Conjugate residuals for (K_sigma + lambda_j I) x_j = y, all lambda_j at once.

    Conjugate residuals minimise ||y - A x|| over the Krylov space, so the
    residual falls monotonically (conjugate gradients minimise the energy norm
    and, on these ill-conditioned kernels, can leave the residual above ||y||
    for many steps).  The kernel product is formed block by block in float32,
    so the snapshots are approximate, as Alg. 1 step 1 allows.  Returns
    (x (N, q) float64, relative residuals of the float32 operator).
    """
    import torch
    N = X.shape[0]
    Xc = (X - X.mean(dim=0)).float()  # centring shrinks the norms the expansion subtracts
    nrm = (Xc * Xc).sum(1)
    lam = torch.as_tensor(np.asarray(lams, dtype=np.float64), device=X.device)
    q = lam.numel()
    y = torch.as_tensor(np.asarray(prob.b, dtype=np.float64), device=X.device)
    inv = 1.0 / (2.0 * sigma * sigma)

    def amul(V):
        out = torch.empty_like(V)
        Vf = V.float()
        for a in range(0, N, block):
            # squared distances by the norm expansion on centred float32 points
            D = (nrm[a:a + block, None] + nrm[None, :] - 2.0 * (Xc[a:a + block] @ Xc.T)).clamp_min_(0.0)
            D.mul_(-inv).exp_()
            out[a:a + block] = (D @ Vf).double()
        return out + lam[None, :] * V

    x = torch.zeros((N, q), dtype=torch.float64, device=X.device)
    r = y[:, None].expand(N, q).clone()
    p = r.clone()
    Ar = amul(r)
    Ap = Ar.clone()
    rAr = (r * Ar).sum(0)
    bn = torch.linalg.vector_norm(y)
    for _ in range(iters):
        alpha = rAr / (Ap * Ap).sum(0)
        x += alpha[None, :] * p
        r -= alpha[None, :] * Ap
        Ar = amul(r)
        rAr_new = (r * Ar).sum(0)
        beta = rAr_new / rAr
        p = r + beta[None, :] * p
        Ap = Ar + beta[None, :] * Ap
        rAr = rAr_new
    res = torch.linalg.vector_norm(y[:, None] - amul(x), dim=0) / bn
    return x, res.cpu().numpy()


def kernel_ridge_basis_torch(prob, X, device="cuda", iters=40):
    """Orthonormal basis of approximate kernel-ridge snapshots on the sqrt(r) x sqrt(r) grid.

    Returns (S_rows (r, N), relative residuals); row k = column k of S.
    """
    import torch
    sig = np.unique(prob.snap_params[:, 0])
    cols, res = [], []
    for sv in sig:
        lams = prob.snap_params[prob.snap_params[:, 0] == sv, 1]
        x, rr = kernel_ridge_cr(prob, X, float(sv), lams, iters=iters)
        cols.append(x)
        res.append(rr)
    Xs = torch.cat(cols, dim=1)
    Q = orthonormalise_torch(Xs)
    return Q.T.contiguous(), np.concatenate(res)
