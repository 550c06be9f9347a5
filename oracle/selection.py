"""Row selection of the oracle: column-pivoted QR on (A(p_sel) S)^T in rounds.

The paper lists CPQR applied to (A(p_i) X)^T as a classic way to pick the
subsampling rows at a representative snapshot point (Sec. 4.3; Alg. 1
step 3).  CPQR on an r x n matrix yields at most r pivots.  For s > r we take
the union idea of Sec. 4.3.2 in rounds: round 1 is plain CPQR; every later
round runs CPQR again on the same matrix with all earlier picks removed; the
last round stops once s indices are held.

Pivot rule (the same on every side that must agree): at each step every
remaining candidate's residual norm ||(I - Q Q^H) v_i||, Q an orthonormal
basis of the candidates already picked in this round, is computed from
scratch in float64; the largest wins and an exact tie goes to the lowest row
index.  Each step's relative gap between the best and the runner-up is
returned so that a disagreement at a near-tie can be told apart from a bug.
"""
from __future__ import annotations

import numpy as np


def cpqr_round(V: np.ndarray, candidates: np.ndarray, k: int):
    """k steps of column-pivoted QR over the rows ``V[candidates]``.

    V is n x r (row i is column i of V^T).  Returns (picked rows, gaps).
    """
    picks = []
    gaps = []
    Q = np.zeros((V.shape[1], 0), dtype=V.dtype)
    alive = np.ones(len(candidates), dtype=bool)
    W = V[candidates]
    for _ in range(k):
        P = W - (W @ Q.conj()) @ Q.T if Q.shape[1] else W.copy()
        norms = np.sqrt((P.real ** 2 + P.imag ** 2).sum(axis=1)) if np.iscomplexobj(P) \
            else np.sqrt((P * P).sum(axis=1))
        norms = np.where(alive, norms, -1.0)
        best = int(np.argmax(norms))  # argmax returns the first of equal maxima
        top = norms[best]
        rest = np.delete(norms, best)
        second = rest.max() if rest.size else -1.0
        gaps.append(float((top - second) / top) if top > 0 else 0.0)
        picks.append(int(candidates[best]))
        alive[best] = False
        rows = V[np.array(picks)]
        Q, _ = np.linalg.qr(rows.T, mode="reduced")  # r x t, spans the picked rows
    return picks, gaps


def cpqr_rows(V: np.ndarray, s: int):
    """s row indices of V (n x r) chosen by CPQR in rounds; returns (J, gaps)."""
    n, r = V.shape
    if not (r <= s <= n):
        raise ValueError("need r <= s <= n")
    chosen: list[int] = []
    gaps: list[float] = []
    while len(chosen) < s:
        cand = np.setdiff1d(np.arange(n), np.array(chosen, dtype=np.int64), assume_unique=False)
        k = min(r, s - len(chosen), cand.size)
        picks, g = cpqr_round(V, cand, k)
        chosen += picks
        gaps += g
    return np.array(chosen, dtype=np.int64), np.array(gaps)


def union_rows(V_list, s_each: int):
    """Union of CPQR picks at several snapshot points (Sec. 4.3.4).

    The variants section proposes choosing rows at t snapshot points and
    keeping every location any of them chose, which oversamples without a
    random draw.  Each V_i = A(p_i) S (n x r) is handled by ``cpqr_rows`` with
    s_each rows; the result lists the distinct rows in order of first
    appearance (point 0's picks first, then what point 1 adds, ...).
    """
    out: list[int] = []
    seen: set[int] = set()
    for V in V_list:
        J, _ = cpqr_rows(np.asarray(V), s_each)
        for j in J.tolist():
            if j not in seen:
                seen.add(j)
                out.append(j)
    return np.array(out, dtype=np.int64)


def nearest_points(params: np.ndarray, points: np.ndarray) -> np.ndarray:
    """Index of the snapshot point closest to each parameter (Sec. 4.3.4).

    The other variant of that section takes, for a new p, the rows chosen at
    its nearest snapshot point.  Distance: Euclidean in the parameter vector;
    an exact tie goes to the lowest index.
    """
    P = np.atleast_2d(np.asarray(params, dtype=np.float64))
    Q = np.atleast_2d(np.asarray(points, dtype=np.float64))
    out = np.empty(P.shape[0], dtype=np.int32)
    for q in range(P.shape[0]):
        d2 = ((Q - P[q]) ** 2).sum(axis=1)
        out[q] = int(np.argmin(d2))
    return out
