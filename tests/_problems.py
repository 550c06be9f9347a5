"""Shared fixtures for the GPU parity tests: workload instance, basis, oracle answers."""
import numpy as np

from oracle import online, problem as oproblem, selection
from workloads import get_config
from workloads import snapshots as wsnap


class Case:
    def __init__(self, name, basis="snapshots", seed_basis=0, rows="cpqr", **kw):
        self.prob = get_config(name, **kw)
        p = self.prob
        if basis == "snapshots":
            self.S = wsnap.basis(p)
        else:  # random orthonormal basis (the online stage does not care where S comes from)
            rng = np.random.default_rng(seed_basis)
            Z = rng.standard_normal((p.n, p.r))
            if p.complex_valued:
                Z = Z + 1j * rng.standard_normal((p.n, p.r))
            self.S = wsnap.orthonormalise(Z)
        if rows == "random":  # the online stage accepts any row set; saves the CPQR at large n
            self.J = np.sort(np.random.default_rng(seed_basis + 1).choice(p.n, p.s, replace=False))
            self.gaps = None
        else:
            V = np.asarray(oproblem.full_matrix(p, p.sel_param) @ self.S)
            self.J, self.gaps = selection.cpqr_rows(V, p.s)

    def oracle_solve(self, params):
        return online.solve_many(self.prob, self.S, self.J, params)

    def kappas(self, params):
        return np.array([online.condition_number(self.prob, self.S, self.J, p) for p in params])


U32 = 2.0 ** -24


def mixed_bound(prob, S, J, params, Yo, rho_o):
    """Distance bound of the mixed solve to the float64 answer, per parameter.

    The float32 factorisation with float64-residual refinement converges to
    the least-squares solution of the perturbed matrix: ~kappa^2 u32 ||r*|| /
    (||M|| ||y||) plus float64 rounding ~kappa u64; 16x that plus 1e-11.
    """
    bounds = []
    bJ = prob.b[np.asarray(J)]
    for prm, y, rr in zip(params, Yo, rho_o):
        M = online.subsampled_matrix(prob, S, J, prm)
        sv = np.linalg.svd(M, compute_uv=False)
        kap = sv[0] / sv[-1]
        rstar = rr * np.linalg.norm(bJ)
        bounds.append(1e-11 + 16 * (kap ** 2 * U32 * rstar / (sv[0] * np.linalg.norm(y)) + kap * 1.1e-16))
    return np.array(bounds)
