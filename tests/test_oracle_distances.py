"""Pins of the distance oracle (oracle/distances.py) to closed forms and
identities that do not come from the oracle itself."""
import itertools

import numpy as np
import pytest

from gen import CFG, config1, structured_cfg
from oracle import distances as D


def cfg_from_dense(T):
    s, d = np.nonzero(T)
    n = T.shape[0]
    return CFG(n, s.astype(np.int32), d.astype(np.int32), T[s, d].astype(np.float64), np.ones((n, 2)))


def test_transition_matrix_sums_duplicates():
    c = CFG(3, np.array([0, 0, 1, 2]), np.array([1, 1, 2, 0]), np.array([0.25, 0.5, 1.0, 2.0]), np.ones((3, 1)))
    T = D.transition_matrix(c)
    assert T.tolist() == [[0, 0.75, 0], [0, 0, 1.0], [2.0, 0, 0]]


def test_resize_identity_and_constant():
    rng = np.random.default_rng(0)
    M = rng.random((6, 6))
    assert np.array_equal(D.resize_bilinear(M, 6), M)
    assert np.allclose(D.resize_bilinear(np.full((4, 4), 2.5), 9), 2.5)
    assert np.allclose(D.resize_bilinear(np.array([[3.0]]), 5), 3.0)


@pytest.mark.parametrize("n,N", [(2, 5), (3, 7), (5, 12), (7, 8), (4, 100)])
def test_resize_reproduces_affine_functions_and_corners(n, N):
    # bilinear interpolation is exact on f(i, j) = a + b i + c j + d i j, sampled on
    # the corner-keeping grid t -> t (n - 1) / (N - 1)
    a, b, c, d = 0.3, -1.2, 2.5, 0.7
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    M = a + b * i + c * j + d * i * j
    R = D.resize_bilinear(M, N)
    u = np.arange(N) * (n - 1) / (N - 1)
    ui, uj = np.meshgrid(u, u, indexing="ij")
    assert np.allclose(R, a + b * ui + c * uj + d * ui * uj, atol=1e-12)
    assert R[0, 0] == M[0, 0] and np.isclose(R[-1, -1], M[-1, -1]) and np.isclose(R[0, -1], M[0, -1])


def test_table1_closed_forms():
    x = np.array([1.0, 0.0, 2.0, 0.0])
    y = np.array([0.0, 1.0, 2.0, 3.0])
    # |x - y| = (1, 1, 0, 3)
    euc, man, mink, jac, cos = D.table1(x, y, p=3)
    assert np.isclose(euc, np.sqrt(11))
    assert man == 5
    assert np.isclose(mink, (1 + 1 + 27) ** (1 / 3))
    # sum x^2 = 5, sum y^2 = 14, sum xy = 4
    assert np.isclose(jac, 11 / (5 + 14 - 4))
    assert np.isclose(cos, 1 - 4 / (np.sqrt(5) * np.sqrt(14)))


def test_table1_identities():
    rng = np.random.default_rng(1)
    for _ in range(20):
        x, y = rng.random(30), rng.random(30)
        d = D.table1(x, y, p=3)
        assert np.isclose(D.table1(x, y, p=2)[2], d[0])  # Minkowski p = 2 is Euclidean
        assert np.isclose(D.table1(x, y, p=1)[2], d[1])  # p = 1 is Manhattan
        assert np.allclose(D.table1(y, x, p=3), d)  # symmetric
        assert np.allclose(D.table1(x, x), 0.0, atol=1e-12)
        assert np.isclose(D.table1(x, 3 * x)[4], 0.0, atol=1e-12)  # cosine of proportional vectors
    z = np.zeros(5)
    assert D.table1(z, z).tolist() == [0, 0, 0, 0, 0]
    assert D.table1(z, np.ones(5))[4] == 1.0


def test_pair_distances_order_and_self():
    w = config1()
    a, b = w.cfgs_a[0], w.cfgs_a[1]
    assert np.allclose(D.pair_distances(a, b), D.pair_distances(b, a))
    assert np.allclose(D.pair_distances(a, a), 0.0, atol=1e-12)


def test_pair_distances_brute_force_on_tiny_graphs():
    # 2-block chain against a 3-block chain: x = resize of [[0, 1], [0, 0]] to 3 x 3 by hand
    A = cfg_from_dense(np.array([[0.0, 1.0], [0.0, 0.0]]))
    B = cfg_from_dense(np.array([[0.0, 0.6, 0.4], [0.0, 0.0, 1.0], [0.0, 0.0, 0.0]]))
    x, y = D.aligned_pair(A, B)
    # grid 0, 0.5, 1 on both axes: rows interpolate [0, 1] and [0, 0]
    want = np.array([[0, 0.5, 1.0], [0, 0.25, 0.5], [0, 0, 0]])
    assert np.allclose(x, want)
    assert np.allclose(y, D.transition_matrix(B))
    diff = (want - y).ravel()
    assert np.isclose(D.pair_distances(A, B)[1], np.abs(diff).sum())


def test_scale01():
    M = np.array([[1.0, 5.0], [3.0, 5.0], [2.0, 5.0]])
    S = D.scale01(M)
    assert S[:, 0].tolist() == [0.0, 1.0, 0.5]
    assert S[:, 1].tolist() == [0.0, 0.0, 0.0]


def test_pins_catch_planted_mistakes():
    # a resize on the other common grid (pixel centres, t -> (t + 0.5) n / N - 0.5,
    # clamped) is not exact on affine functions at the corners
    n, N = 4, 9
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    M = 1.0 + 2.0 * i - 0.5 * j

    def centre_grid(M, N):
        n = M.shape[0]
        f = np.clip((np.arange(N) + 0.5) * n / N - 0.5, 0, n - 1)
        i0 = np.minimum(np.floor(f).astype(int), n - 2)
        a = f - i0
        rows = (1 - a)[:, None] * M[i0] + a[:, None] * M[i0 + 1]
        return (1 - a)[None, :] * rows[:, i0] + a[None, :] * rows[:, i0 + 1]

    u = np.arange(N) * (n - 1) / (N - 1)
    want = 1.0 + 2.0 * u[:, None] - 0.5 * u[None, :]
    assert np.allclose(D.resize_bilinear(M, N), want)
    assert not np.allclose(centre_grid(M, N), want)
    # a Manhattan without the absolute value, or a Jaccard without the cross term,
    # fails the closed forms
    x, y = np.array([1.0, 0.0, 2.0, 0.0]), np.array([0.0, 1.0, 2.0, 3.0])
    assert np.sum(x - y) != D.table1(x, y)[1]
    assert not np.isclose(np.sum((x - y) ** 2) / (x @ x + y @ y), D.table1(x, y)[3])
