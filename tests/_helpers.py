"""Shared test helpers: tolerance checks and greedy-margin analysis."""
import numpy as np

import oracle

# Tolerances (normalised X entries and graph scores; FP32 GPU vs FP64 oracle)
ATOL_X = 1e-5
ATOL_S = 1e-5
TIE_EPS = 1e-6  # matchings compared index by index when every greedy decision wins by more than this


def greedy_margin(X: np.ndarray) -> float:
    """Smallest gap between each greedy pick and its best live competitor in
    the same row or column (inf if there is none)."""
    m, _ = oracle.greedy_match(X)
    n1, n2 = X.shape
    picks = sorted([(X[i, m[i]], i, int(m[i])) for i in range(n1) if m[i] >= 0], key=lambda t: (-t[0], t[1], t[2]))
    alive_r = np.ones(n1, bool)
    alive_c = np.ones(n2, bool)
    gap = np.inf
    for v, i, j in picks:
        row = X[i, alive_c].copy()
        col = X[alive_r, j].copy()
        # remove the pick itself from both
        cj = np.flatnonzero(alive_c)
        ri = np.flatnonzero(alive_r)
        row = row[cj != j]
        col = col[ri != i]
        comp = np.concatenate([row, col])
        if comp.size:
            gap = min(gap, v - comp.max())
        alive_r[i] = False
        alive_c[j] = False
    return gap


def valid_matching(match: np.ndarray, n1: int, n2: int) -> bool:
    used = match[match >= 0]
    return (len(used) == min(n1, n2) and len(set(used.tolist())) == len(used)
            and (used < n2).all() and ((match >= -1).all()))


def eps_greedy(Xg: np.ndarray, Xr: np.ndarray, match: np.ndarray, eps: float) -> bool:
    """The matching is what greedy gives on some matrix within eps/2 of Xr:
    replayed in the GPU's own pick order (its values Xg descending), every
    pick is within eps of the largest live entry of Xr."""
    n1, n2 = Xr.shape
    picks = sorted([(Xg[i, match[i]], i, int(match[i])) for i in range(n1) if match[i] >= 0],
                   key=lambda t: (-t[0], t[1], t[2]))
    alive_r = np.ones(n1, bool)
    alive_c = np.ones(n2, bool)
    for _, i, j in picks:
        if not (alive_r[i] and alive_c[j]):
            return False
        best = Xr[np.ix_(alive_r, alive_c)].max()
        if Xr[i, j] < best - eps:
            return False
        alive_r[i] = False
        alive_c[j] = False
    return True
