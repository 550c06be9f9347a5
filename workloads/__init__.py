"""Seeded synthetic workloads for the SubApSnap online stage.

This module is shared by the CPU oracle and the CUDA path.  It defines the
problems (operators A(p) = sum_k theta_k(p) A_k, right-hand sides, parameter
draws, kernel-regression data) and nothing of the method's own arithmetic:
no subsampled least squares, no assembly of A(p)_J S, no row selection, no
reconstruction.  Snapshot solutions x(p_i) are inputs of the online stage and
are produced here by generic sparse solvers (see ``workloads.snapshots``).
"""
from .configs import CONFIGS, get_config  # noqa: F401
