"""CPU oracle for the SubApSnap online stage (test infrastructure only).

This package is the slow, plain, float64 / complex128 statement of what the
method computes, written from the paper (SubApSnap, arXiv 2510.04825).  It is
used by the test-suite, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``; nothing in the product library imports it, and it shares
no code with the CUDA path.  The only module both sides use is ``workloads``
(seeded problem generators).

Modules
  problem    theta(p), explicit rows of A(p), full A(p)            (Sec. 3, 3.1)
  linalg     Thomas solver, Householder least squares               (Alg. 1 step 4)
  snapshots  snapshot solves and orthonormalisation                 (Alg. 1 steps 1-2)
  selection  column-pivoted QR on (A(p_sel) S)^T, in rounds          (Alg. 1 step 3, Sec. 4.3)
  online     subsampled LS, reconstruction, QoI, residuals          (Alg. 1 step 4, Sec. 5.2.2)
  krr        Gaussian-kernel rows for kernel ridge regression       (Sec. 5.3)
  mlp        float64 MLP forward/backward/Adam for the surrogate    (no counterpart in the paper)

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: closed forms (s = n gives the full least squares, s = r interpolates,
A = I gives DEIM, p at a snapshot recovers x(p)), Lemma 4.1's inequalities,
brute force in extended precision, and library routines for special cases.
The MLP's gradients are pinned by central finite differences; its place in the
method is not from the paper.
"""
