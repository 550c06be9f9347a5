"""Shared fixtures for the GPU parity tests: workload instance, basis, oracle answers."""
import numpy as np

from oracle import online, problem as oproblem, selection
from workloads import get_config
from workloads import snapshots as wsnap


class Case:
    def __init__(self, name, basis="snapshots", seed_basis=0, **kw):
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
        V = np.asarray(oproblem.full_matrix(p, p.sel_param) @ self.S)
        self.J, self.gaps = selection.cpqr_rows(V, p.s)

    def oracle_solve(self, params):
        return online.solve_many(self.prob, self.S, self.J, params)

    def kappas(self, params):
        return np.array([online.condition_number(self.prob, self.S, self.J, p) for p in params])
