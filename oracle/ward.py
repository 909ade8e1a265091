"""FP64 CPU oracle for Ward clustering of CFGs by their similarity profiles.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package.  The product
path never calls it, and this module imports nothing from the product path.

Sec. 5.3 groups kernels with Ward's minimum-variance method, whose initial
cluster distances are squared Euclidean distances between points,
``d_ij = |X_i - X_j|^2``.  The paper does not say which vector a kernel's point
is; the reading here: CFG i is the point ``X_i = S[i, :]``, its row of the
all-pairs graph-score matrix (its similarity profile against every CFG of the
set, the diagonal holding its self-score).

``linkage`` returns scipy's linkage matrix for those points (a library step:
``scipy.cluster.hierarchy.linkage(X, "ward")``): row k merges clusters
``Z[k, 0] < Z[k, 1]`` (ids below n are points, ``n + k`` the cluster made at
step k) at height ``Z[k, 2]`` with ``Z[k, 3]`` points.  ``linkage_naive``
restates Ward's criterion directly -- merge the two clusters whose union
raises the total within-cluster sum of squares least,
``dESS(A, B) = |A| |B| / (|A| + |B|) |c_A - c_B|^2`` -- and is the pin: its
heights are ``sqrt(2 dESS)``.
"""
from __future__ import annotations

import numpy as np


def score_matrix(n: int, pairs, scores, symmetric: bool = True) -> np.ndarray:
    """Dense ``n x n`` matrix with ``S[a, b] = score`` of pair (a, b) (and
    ``S[b, a]`` too when ``symmetric``); entries of absent pairs are 0."""
    S = np.zeros((n, n))
    for (a, b), s in zip(np.asarray(pairs), np.asarray(scores, dtype=np.float64)):
        S[int(a), int(b)] = s
        if symmetric:
            S[int(b), int(a)] = s
    return S


def linkage(X: np.ndarray) -> np.ndarray:
    from scipy.cluster.hierarchy import linkage as _linkage

    return _linkage(np.asarray(X, dtype=np.float64), method="ward")


def linkage_naive(X: np.ndarray) -> np.ndarray:
    """Ward by exhaustive search over cluster pairs (O(n^3) per merge; small n).
    Ties: the pair with the smallest (smaller id, larger id)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    members = {i: [i] for i in range(n)}
    Z = np.zeros((n - 1, 4))
    for k in range(n - 1):
        ids = sorted(members)
        best = None
        for ia, a in enumerate(ids):
            ca = X[members[a]].mean(axis=0)
            for b in ids[ia + 1:]:
                cb = X[members[b]].mean(axis=0)
                na, nb = len(members[a]), len(members[b])
                dess = na * nb / (na + nb) * float(np.sum((ca - cb) ** 2))
                if best is None or dess < best[0]:
                    best = (dess, a, b)
        dess, a, b = best
        members[n + k] = members.pop(a) + members.pop(b)
        Z[k] = [a, b, np.sqrt(2.0 * dess), len(members[n + k])]
    return Z
