"""Pins of the subsampling variants of Sec. 4.3.4: union of pivot sets, nearest point.

The hand examples have rows along the coordinate axes, so every CPQR step can
be worked out on paper: the largest row norm wins, and projecting out a unit
axis zeroes that coordinate of every remaining row.
"""
import numpy as np

from oracle import online, problem, selection, snapshots
from workloads import get_config

# point 1: rows 3 (|.|=5) then 0 (3 once e_2 is removed); round 2 adds row 2 (|.|=2)
V1 = np.array([[3, 0], [0, 1], [2, 0], [0, 5], [0.1, 0.1], [1, 0.5]], dtype=float)
# point 2: rows 1 (|.|=4) then 5 (3 once e_1 is removed)
V2 = np.array([[0, 0.5], [4, 0], [0, 2], [1, 1], [0, 0], [0, 3]], dtype=float)


def test_cpqr_hand_examples():
    np.testing.assert_array_equal(selection.cpqr_rows(V1, 2)[0], [3, 0])
    np.testing.assert_array_equal(selection.cpqr_rows(V1, 3)[0], [3, 0, 2])
    np.testing.assert_array_equal(selection.cpqr_rows(V2, 2)[0], [1, 5])


def test_union_hand_example():
    np.testing.assert_array_equal(selection.union_rows([V1, V2], 2), [3, 0, 1, 5])
    # a repeated point adds nothing; order follows first appearance
    np.testing.assert_array_equal(selection.union_rows([V2, V1, V2], 2), [1, 5, 3, 0])
    np.testing.assert_array_equal(selection.union_rows([V1, V2], 3)[:3], [3, 0, 2])


def test_union_of_one_point_is_cpqr_and_contains_every_point():
    prob = get_config("reaction_diffusion_1d", n=600, r=8, s=16, m=10)
    S = snapshots.orthonormal_basis(snapshots.snapshot_matrix(prob))
    pts = prob.snap_params[[0, 3, 7]]
    Vs = [np.asarray(problem.full_matrix(prob, pt) @ S) for pt in pts]
    np.testing.assert_array_equal(selection.union_rows(Vs[:1], prob.r), selection.cpqr_rows(Vs[0], prob.r)[0])
    U = selection.union_rows(Vs, prob.r)
    assert len(set(U.tolist())) == len(U)
    assert prob.r <= len(U) <= 3 * prob.r
    for V in Vs:
        assert set(selection.cpqr_rows(V, prob.r)[0].tolist()) <= set(U.tolist())
    # each union row set oversamples: s = |U| >= r, and at the chosen points
    # the subsampled solve is exact (the snapshot lies in span S)
    for pt in pts:
        y, rho = online.solve_one(prob, S, U, pt)
        assert rho < 1e-8


def test_nearest_points_hand_example():
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    P = np.array([[0.4, 0.1], [0.6, 0.0], [0.5, 0.0], [0.0, 1.2], [10.0, 10.0]])
    # (0.5, 0) is equidistant from points 0 and 1: the lower index wins;
    # (10, 10): 181 to point 1, 164 to point 2
    np.testing.assert_array_equal(selection.nearest_points(P, pts), [0, 1, 0, 2, 2])
    np.testing.assert_array_equal(selection.nearest_points(np.array([[3.0]]), np.array([[1.0], [4.0], [2.0]])), [1])
