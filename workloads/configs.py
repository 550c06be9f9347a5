"""The five synthetic workloads of the online stage, with seeded draws.

Each ``make_*`` builds a problem at a given size; the full sizes are the
defaults.  Random draws use ``numpy.random.default_rng(seed)`` (PCG64) in the
order documented per function, so a smaller instance is a different draw.

Parameter conventions (what the online stage receives per new parameter):
  reaction_diffusion_1d : p in [0, 10]            A(p) = L + p D
  diffusion_2d          : p in [0, 1]^4           A(p) = A_0 + sum_k p_k A_k
  kernel_ridge          : p = (sigma, lambda)     A(p) = K_sigma + lambda I
  transfer_function     : p = omega, s = i omega  A(s) = s E - A_0
  delay_system          : p = (omega, tau)        A = i omega I - A_0 - e^{i omega tau} A_1
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import operators as ops


@dataclass
class AffineProblem:
    """A(p) = sum_k theta_k(p) A_k with a constant right-hand side b.

    ``theta_rule`` names how theta(p) is formed from a parameter vector:
      "linear": theta = (1, p_1, ..., p_d)        (real)
      "pencil": theta = (-1, i*omega) for (A_0, E) (complex; p = omega)
      "delay":  theta = (i omega, -1, -e^{i omega tau}) for (I, A_0, A_1)
                (complex; p = (omega, tau))
    """
    name: str
    n: int
    blocks: list
    theta_rule: str
    b: np.ndarray
    r: int
    s: int
    snap_params: np.ndarray
    sel_param: np.ndarray
    test_params: np.ndarray
    complex_valued: bool = False
    c: np.ndarray | None = None      # QoI vector (None: no QoI)
    qoi_kind: str | None = None      # "transpose" (c^T x) or "mean" (1^T x / n)
    grid: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return len(self.blocks)

    @property
    def dp(self) -> int:
        return self.test_params.shape[1]


@dataclass
class KernelProblem:
    """A(sigma, lambda) = K_sigma + lambda I on points X (N x d), b = targets."""
    name: str
    n: int
    X: np.ndarray
    b: np.ndarray
    r: int
    s: int
    snap_params: np.ndarray
    sel_param: np.ndarray
    test_params: np.ndarray
    complex_valued: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def dp(self) -> int:
        return 2


def chebyshev_points(a: float, b: float, r: int) -> np.ndarray:
    """Chebyshev points of the second kind (extrema, endpoints included) on [a, b]."""
    j = np.arange(r)
    return 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * j / (r - 1))


def make_reaction_diffusion_1d(n=4096, r=20, s=40, m=1000, seed=0) -> AffineProblem:
    """1-D reaction-diffusion: A(p) = L + p diag(d), p in [0, 10], b = ones.

    Draw order: d ~ U[0,1]^n, then the m test parameters ~ U[0,10].
    Snapshots at r Chebyshev points of [0, 10]; selection at p = 5.
    """
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.0, 1.0, n)
    test = rng.uniform(0.0, 10.0, m)
    L = ops.tridiag_laplacian(n)
    D = sp.diags(d, 0, format="csr")
    return AffineProblem(
        name="reaction_diffusion_1d", n=n, blocks=[L, D], theta_rule="linear",
        b=np.ones(n), r=r, s=s, snap_params=chebyshev_points(0.0, 10.0, r)[:, None],
        sel_param=np.array([5.0]), test_params=test[:, None], grid=(n,),
        meta={"d": d},
    )


def make_diffusion_2d(N=1024, r=60, s=120, m=4096, nbump=4, width=0.1, seed=0,
                      name="diffusion_2d") -> AffineProblem:
    """2-D diffusion -div(a(x;p) grad u) = 1 on the unit square, Dirichlet.

    a(x;p) = 1 + sum_k p_k psi_k(x), psi_k Gaussian bumps of width 0.1.
    Draw order: centres ~ U[0.1,0.9]^2 (nbump x 2), snapshot parameters
    ~ U[0,1]^4 (r x 4), test parameters ~ U[0,1]^4 (m x 4).
    Selection at the median point p = (0.5, 0.5, 0.5, 0.5).
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, (nbump, 2))
    snap = rng.uniform(0.0, 1.0, (r, nbump))
    test = rng.uniform(0.0, 1.0, (m, nbump))
    h = 1.0 / (N + 1)
    ones_x = np.ones((N + 1, N)); ones_y = np.ones((N, N + 1))
    blocks = [ops.diffusion_2d(N, ones_x, ones_y, h)]
    faces = []
    for k in range(nbump):
        ax, ay = ops.gaussian_bump_faces(N, centres[k], width)
        faces.append((ax, ay))
        blocks.append(ops.diffusion_2d(N, ax, ay, h))
    n = N * N
    return AffineProblem(
        name=name, n=n, blocks=blocks, theta_rule="linear", b=np.ones(n), r=r, s=s,
        snap_params=snap, sel_param=np.full(nbump, 0.5), test_params=test,
        c=np.full(n, 1.0 / n), qoi_kind="mean", grid=(N, N),
        meta={"centres": centres, "width": width, "h": h, "faces": faces},
    )


def make_surrogate_diffusion_2d(N=4096, r=60, s=120, m=65536, seed=0) -> AffineProblem:
    """The 2-D diffusion workload at 4096 x 4096 (learned-surrogate workload)."""
    return make_diffusion_2d(N=N, r=r, s=s, m=m, seed=seed, name="surrogate_diffusion_2d")


def make_transfer_function(N=100, r=80, s=200, m=16384, seed=0) -> AffineProblem:
    """Transfer function H(i w) = c^T (i w E - A_0)^{-1} b on an N^3 heat grid.

    A_0 = h^-2 * 7-point Laplacian, E = diag(e), e ~ U[0.5, 1.5].
    Draw order: e (n), b ~ N(0,1)^n, c ~ N(0,1)^n.  Snapshots at r
    log-spaced omega in [1e-2, 1e4]; test omega = logspace(-2, 4, m);
    selection at omega = 10 (log-midpoint).
    """
    rng = np.random.default_rng(seed)
    n = N ** 3
    e = rng.uniform(0.5, 1.5, n)
    b = rng.standard_normal(n)
    c = rng.standard_normal(n)
    A0 = ops.heat_3d(N)
    E = sp.diags(e, 0, format="csr")
    return AffineProblem(
        name="transfer_function", n=n, blocks=[A0, E], theta_rule="pencil", b=b.astype(np.complex128),
        r=r, s=s, snap_params=np.logspace(-2, 4, r)[:, None], sel_param=np.array([10.0]),
        test_params=np.logspace(-2, 4, m)[:, None], complex_valued=True, c=c,
        qoi_kind="transpose", grid=(N, N, N), meta={"e": e},
    )


def make_kernel_ridge(N=200_000, d=8, ncomp=10, nfreq=5, r=100, s=300, m=2048, seed=0) -> KernelProblem:
    """Kernel ridge regression (K_sigma + lambda I) x = y on a Gaussian mixture.

    Draw order: component labels (N), component means ~ N(0, 4 I) (ncomp x d),
    points = mean + sqrt(0.5) N(0, I), frequencies w_j ~ N(0, I) (nfreq x d),
    noise ~ N(0,1) (N), test sigma ~ U[0.5, 2] (m), test log10(lambda) ~
    U[-4, -1] (m).  Snapshots on a sqrt(r) x sqrt(r) grid: sigma linear in
    [0.5, 2], lambda log-spaced in [1e-4, 1e-1].  Selection at the grid's
    median point (sigma, lambda) = (1.25, 10^-2.5).
    """
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, ncomp, N)
    means = 2.0 * rng.standard_normal((ncomp, d))
    X = means[labels] + np.sqrt(0.5) * rng.standard_normal((N, d))
    W = rng.standard_normal((nfreq, d))
    noise = rng.standard_normal(N)
    y = np.sin(X @ W.T).sum(axis=1) + 0.1 * noise
    sig = rng.uniform(0.5, 2.0, m)
    lam = 10.0 ** rng.uniform(-4.0, -1.0, m)
    g = int(round(np.sqrt(r)))
    sg = np.linspace(0.5, 2.0, g)
    lg = np.logspace(-4, -1, g)
    snap = np.array([(a, b) for a in sg for b in lg])
    if snap.shape[0] != r:
        raise ValueError("kernel ridge snapshots need r to be a perfect square")
    return KernelProblem(
        name="kernel_ridge", n=N, X=X, b=y, r=r, s=s, snap_params=snap,
        sel_param=np.array([1.25, 10.0 ** -2.5]), test_params=np.stack([sig, lam], 1),
        meta={"d": d},
    )


def make_delay_system(n=10_000_000, r=24, s=48, m=5000, tau=0.1, kappa=2.1,
                      seed=0) -> AffineProblem:
    """Delay system H(p) = c^T (p I - A_0 - e^{tau p} A_1)^{-1} b on the imaginary axis
    p = i omega (Sec. 5.2.3, Table 4): A_1 = (T - kappa I)/tau, A_0 = 3 A_1, tau = 0.1,
    kappa = 2.1.  Draw order: b ~ N(0,1)^n, c ~ N(0,1)^n (every row of T sums to 2,
    so a constant b would be an eigenvector of A(p) and every snapshot a multiple
    of it).  Snapshots at r = 24 log-spaced omega in [1e-2, 1e3] (the snapshot set's
    numerical rank is ~26 at 1e-14: more snapshots add rounding noise to S); test omega =
    logspace(-2, 3, m) (endpoints shared with the snapshots); selection at the
    log-midpoint omega = 10^0.5.  Parameters carry tau as their second entry.
    """
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n)
    c = rng.standard_normal(n)
    I, A0, A1 = ops.delay_blocks(n, tau, kappa)
    snap = np.logspace(-2, 3, r)
    test = np.logspace(-2, 3, m)
    return AffineProblem(
        name="delay_system", n=n, blocks=[I, A0, A1], theta_rule="delay",
        b=b.astype(np.complex128), r=r, s=s,
        snap_params=np.stack([snap, np.full(r, tau)], 1),
        sel_param=np.array([10.0 ** 0.5, tau]),
        test_params=np.stack([test, np.full(m, tau)], 1), complex_valued=True,
        c=c, qoi_kind="transpose", meta={"tau": tau, "kappa": kappa},
    )


CONFIGS = {
    "reaction_diffusion_1d": make_reaction_diffusion_1d,
    "diffusion_2d": make_diffusion_2d,
    "kernel_ridge": make_kernel_ridge,
    "transfer_function": make_transfer_function,
    "delay_system": make_delay_system,
    "surrogate_diffusion_2d": make_surrogate_diffusion_2d,
}


def get_config(name: str, **overrides):
    return CONFIGS[name](**overrides)
