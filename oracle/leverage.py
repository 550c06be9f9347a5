"""Leverage-score row sampling with weights, and the residual estimate it gives
(oracle; test infrastructure only, never imported by the library).

Sec. 4.3.2 lists leverage-score sampling among the ways to choose the rows J:
rows are drawn with probability proportional to the squared row norms of Q,
where A(p_sel) X = QR, and with oversampling (s > r) each kept row carries the
weight 1/sqrt(s pi_i) (the footnote of Sec. 4.3.2), so that the sketch S
satisfies E[S^T S] = I.  Sec. 4.3.3 samples on span([B, b]) with B = A(p_sel) X;
then ||S (B c - b)|| estimates ||B c - b|| within factors (1 - eps, 1 + eps),
eps ~ r log(r) / s, with high probability at p_sel (a heuristic at other p).

Readings (the paper leaves them open):
  * sampling is with replacement, by inverse CDF of the normalised scores on
    caller-supplied uniforms u in [0, 1): with C the running sums of the scores
    in row order (float64) and total = C[-1], draw t is the first row i with
    C[i] / total > u_t;
  * a row drawn k times is kept once with weight sqrt(k / (s pi_i)), the same
    least-squares objective as k weighted copies;
  * the band uses eps = min(r log(r) / s, 1/2) of Sec. 4.3.3 (r >= 2), r the number of
    columns of B.
"""
from __future__ import annotations

import numpy as np


def leverage_scores(V: np.ndarray) -> np.ndarray:
    """Squared row norms of Q for V = QR (thin QR, full column rank)."""
    Q, _ = np.linalg.qr(V, mode="reduced")
    return (Q.real ** 2 + Q.imag ** 2).sum(axis=1) if np.iscomplexobj(Q) else (Q * Q).sum(axis=1)


def sample_rows(scores: np.ndarray, s: int, u: np.ndarray):
    """(J sorted, weights) from s inverse-CDF draws on the uniforms u (length s)."""
    run = np.cumsum(np.asarray(scores, dtype=np.float64))  # running sums in row order
    total = run[-1]
    pi = scores / total
    cdf = run / total
    draws = []
    for ut in np.asarray(u, dtype=np.float64):
        i = int(np.searchsorted(cdf, ut, side="right"))  # first i with cdf[i] > ut
        draws.append(min(i, len(pi) - 1))
    J, counts = np.unique(np.array(draws, dtype=np.int64), return_counts=True)
    w = np.sqrt(counts / (s * pi[J]))
    return J, w


def band_epsilon(r: int, s: int) -> float:
    """eps of the residual band (1 -/+ eps) ||S(Bc - b)|| of Sec. 4.3.3."""
    return float(min(r * np.log(max(r, 2)) / s, 0.5))
