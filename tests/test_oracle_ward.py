"""Pins of the Ward oracle (oracle/ward.py): scipy's linkage against a direct
restatement of Ward's criterion, and hand cases."""
import numpy as np
import pytest

from oracle import ward as W

pytest.importorskip("scipy")


def test_linkage_equals_ward_criterion_on_random_points():
    rng = np.random.default_rng(11)
    for n, d in [(2, 1), (3, 2), (6, 3), (9, 4), (14, 5)]:
        X = rng.random((n, d))
        Z = W.linkage(X)
        Zn = W.linkage_naive(X)
        assert np.allclose(Z[:, 2], Zn[:, 2], atol=1e-12)
        assert np.array_equal(Z[:, 3], Zn[:, 3])
        for k in range(n - 1):
            assert set(Z[k, :2].astype(int)) == set(Zn[k, :2].astype(int))


def test_hand_case_two_groups():
    # points 0, 1 at 0 and 1 on a line; 2, 3 at 10 and 12
    X = np.array([[0.0], [1.0], [10.0], [12.0]])
    Z = W.linkage(X)
    # first merge {0, 1}: dESS = 1/2 * 1 -> height 1; then {2, 3}: height 2
    assert set(Z[0, :2]) == {0, 1} and np.isclose(Z[0, 2], 1.0)
    assert set(Z[1, :2]) == {2, 3} and np.isclose(Z[1, 2], 2.0)
    # last merge: centroids 0.5 and 11, sizes 2 and 2 -> dESS = 1 * 10.5^2 -> height sqrt(2) * 10.5
    assert np.isclose(Z[2, 2], np.sqrt(2.0) * 10.5) and Z[2, 3] == 4


def test_heights_are_monotone_and_score_matrix():
    rng = np.random.default_rng(3)
    X = rng.random((20, 6))
    Z = W.linkage(X)
    assert np.all(np.diff(Z[:, 2]) >= -1e-12)  # Ward has no inversions
    S = W.score_matrix(3, [(0, 1), (1, 2), (0, 0)], [0.5, 0.25, 1.0])
    assert S.tolist() == [[1.0, 0.5, 0.0], [0.5, 0.0, 0.25], [0.0, 0.25, 0.0]]


def test_planted_mistake_unweighted_centroid_distance_is_caught():
    # merging by the plain centroid distance (without the |A||B|/(|A|+|B|) weight)
    # gives a different merge sequence on this seeded set; the Ward criterion does not
    X = np.random.default_rng(5).random((6, 2))
    members = {i: [i] for i in range(6)}
    order = []
    for k in range(5):
        ids = sorted(members)
        _, a, b = min((float(np.linalg.norm(X[members[a]].mean(0) - X[members[b]].mean(0))), a, b)
                      for i, a in enumerate(ids) for b in ids[i + 1:])
        members[6 + k] = members.pop(a) + members.pop(b)
        order.append((a, b))
    ward = [tuple(sorted(int(v) for v in z[:2])) for z in W.linkage(X)]
    assert ward == [tuple(sorted(int(v) for v in z[:2])) for z in W.linkage_naive(X)]
    assert ward != order
