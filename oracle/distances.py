"""FP64 CPU oracle for the paper's element-wise CFG distances.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package.  The product
path never calls it, and this module imports nothing from the product path.

What it computes, with the passage each step follows (paper arXiv:1707.02423):

1. Transition matrix of a CFG: the dense ``n x n`` matrix ``T[s, d]`` = weight
   of edge ``s -> d`` (Sec. 3.1, transition probabilities; duplicate edges add
   up).
2. Resizing (Sec. 4 and 4.1): the two matrices are brought to the same size by
   bilinear interpolation of the smaller one up to ``N = max(n1, n2)``.  The
   paper names bilinear interpolation (linear interpolation along rows, then
   along columns) but not its sampling grid; the reading here keeps the
   corners: output index ``r`` samples the source at ``r (n - 1) / (N - 1)``
   (a 1 x 1 source stays constant).  When ``n1 == n2`` nothing is resized.
3. The five element-wise distances of Table 1 between the flattened
   ``N x N`` matrices ``x`` (resized smaller graph) and ``y`` (larger graph):
   Euclidean ``sqrt(sum (x - y)^2)``, Manhattan ``sum |x - y|``, Minkowski
   ``(sum |x - y|^p)^(1/p)``, Jaccard
   ``sum (x - y)^2 / (sum x^2 + sum y^2 - sum x y)`` and Cosine
   ``1 - sum x y / (|x| |y|)``.  Zero denominators (both matrices empty of
   edges) give 0 for Jaccard, and Cosine gives 0 if both norms are 0 and 1 if
   exactly one is.
4. Scaling (Sec. 5.2): each distance is min-max scaled to [0, 1] over the set
   of compared pairs (0 = strongest similarity); a constant column scales to 0.

Pins: tests/test_oracle_distances.py (closed forms, affine-exactness of the
bilinear resize, identities between the distances).
"""
from __future__ import annotations

import numpy as np

NAMES = ("euclidean", "manhattan", "minkowski", "jaccard", "cosine")


def transition_matrix(cfg) -> np.ndarray:
    """Dense ``T[s, d] = sum of w_e over edges s -> d`` (Sec. 3.1)."""
    T = np.zeros((cfg.n, cfg.n), dtype=np.float64)
    for s, d, w in zip(np.asarray(cfg.src), np.asarray(cfg.dst), np.asarray(cfg.w, dtype=np.float64)):
        T[int(s), int(d)] += w
    return T


def resize_bilinear(M: np.ndarray, N: int) -> np.ndarray:
    """Bilinear resize of a square ``n x n`` matrix to ``N x N`` (corner-keeping
    grid, see the module docstring): linear interpolation along the rows, then
    along the columns."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    if n == 1:
        return np.full((N, N), M[0, 0])
    if N == 1:
        return M[:1, :1].copy()

    def coords(k):
        f = k * (n - 1) / (N - 1)
        i0 = min(int(np.floor(f)), n - 2)
        return i0, f - i0

    rows = np.empty((N, n))
    for r in range(N):
        i0, a = coords(r)
        rows[r] = (1 - a) * M[i0] + a * M[i0 + 1]
    out = np.empty((N, N))
    for c in range(N):
        j0, b = coords(c)
        out[:, c] = (1 - b) * rows[:, j0] + b * rows[:, j0 + 1]
    return out


def aligned_pair(cfg_a, cfg_b) -> tuple[np.ndarray, np.ndarray]:
    """``(x, y)``: the smaller graph's transition matrix resized to the larger
    size, and the larger graph's (Sec. 4); for equal sizes A is x."""
    Ta, Tb = transition_matrix(cfg_a), transition_matrix(cfg_b)
    if cfg_a.n <= cfg_b.n:
        return resize_bilinear(Ta, cfg_b.n), Tb
    return resize_bilinear(Tb, cfg_a.n), Ta


def table1(x: np.ndarray, y: np.ndarray, p: float = 3.0) -> np.ndarray:
    """The five Table 1 distances of two equal-shape arrays, in NAMES order."""
    x = np.asarray(x, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    d = np.abs(x - y)
    sxx, syy, sxy = float(x @ x), float(y @ y), float(x @ y)
    euc = float(np.sqrt(np.sum(d * d)))
    man = float(np.sum(d))
    mink = float(np.sum(d ** p) ** (1.0 / p))
    den = sxx + syy - sxy
    jac = float(np.sum(d * d) / den) if den > 0 else 0.0
    nx, ny = np.sqrt(sxx), np.sqrt(syy)
    if nx > 0 and ny > 0:
        cos = 1.0 - sxy / (nx * ny)
    else:
        cos = 0.0 if (nx == 0 and ny == 0) else 1.0
    return np.array([euc, man, mink, jac, cos])


def pair_distances(cfg_a, cfg_b, p: float = 3.0) -> np.ndarray:
    x, y = aligned_pair(cfg_a, cfg_b)
    return table1(x, y, p)


def scale01(D: np.ndarray) -> np.ndarray:
    """Min-max scaling of each column of ``D`` ([pairs, measures]) to [0, 1]."""
    D = np.asarray(D, dtype=np.float64)
    lo, hi = D.min(axis=0), D.max(axis=0)
    span = hi - lo
    out = np.zeros_like(D)
    ok = span > 0
    out[:, ok] = (D[:, ok] - lo[ok]) / span[ok]
    return out


def run_pairs(cfgs_a, cfgs_b, pairs, p: float = 3.0, scale: bool = False) -> np.ndarray:
    D = np.array([pair_distances(cfgs_a[a], cfgs_b[b], p) for a, b in pairs]).reshape(-1, 5)
    return scale01(D) if scale else D
