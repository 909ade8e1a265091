"""FP64 CPU oracle for the CFG similarity measure (IsoRank family).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package.  The product
path (the C-ABI library and its Python binding) never calls it, and this
package imports nothing from the product path.

Plain, slow and meant to be read against the paper.  Every array is float64.
Sparse matrix products (scipy) and a sort are the only library steps.

What it computes, with the passage each step follows (paper arXiv:1707.02423):

1. Attribute term ``E`` -- Table 1, "Cos" row, used in similarity form
   ``E_ij = <a_i, b_j>_w / (|a_i|_w |b_j|_w)`` with per-feature weights
   ``w = omega`` (``<x, y>_w = sum_f omega_f x_f y_f``), on the block attributes
   the paper matches on (Sec. 1 and 3.1: instruction operations executed,
   registers allocated, block frequencies).  ``E_ij = 0`` when either norm is 0.
2. Restart term ``Ehat = E / |E|_F`` (uniform ``1/sqrt(n1 n2)`` when ``|E|_F = 0``);
   ``X_0 = Ehat``.
3. Iteration (Table 1, "Iso" row ``(I - alpha Q x P) x`` with ``x`` read as the
   Kronecker product of the two graphs' weighted adjacency operators, after the
   IsoRank method the paper cites in Sec. 2 and Sec. 4.2), for k = 0..K-1::

       Z_k     = 1/2 (W_A X_k W_B^T + W_A^T X_k W_B)     successor + predecessor pairs
       Y_{k+1} = alpha Z_k + (1 - alpha) Ehat
       X_{k+1} = Y_{k+1} / |Y_{k+1}|_F                   (skipped when normalize=False)

   ``W_A[s, d]`` is the weight of edge ``s -> d``: a branch (transition)
   probability (Sec. 3.1, "Transition probability"); duplicate edges add up.
   Without the per-step renormalisation the fixed point solves
   ``(I - alpha M) vec X = (1 - alpha) vec Ehat`` with
   ``M = 1/2 (W_B kron W_A + W_B^T kron W_A^T)`` (column-major vec), the
   Table 1 linear system.  The paper gives no iteration count or stopping
   rule; K = 40 iterations, no early stop.
4. Node matching: greedy on ``X_K`` -- repeatedly take the largest remaining
   entry (ties: smaller row index, then smaller column index), delete its row
   and column, until ``min(n1, n2)`` pairs are taken.  The paper states
   subgraph matching from the measure (Sec. 1, 4, 5.2) but not the procedure.
5. Graph score ``s = sum of X_K over the matched entries`` -- the paper reports
   IsoRank scores between 1.00 and 1.30 (Sec. 5.2, Fig. 5), so the score is an
   unnormalised sum, higher meaning more similar.
6. Reverse mode of 1-5 with the matching frozen: gradients of ``s`` with
   respect to every edge weight of both graphs and to ``omega``.

Parity pins (tests/test_oracle_pins.py) tie each step to something other than
this file: hand-computed values, the Kronecker linear system solved by
numpy.linalg.solve, brute-force matching, symmetry and relabelling
invariants, and central finite differences for the gradient.  The paper prints
no output value of the measure for any concrete input, so no pin comes from a
printed result.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------- graphs
def adjacency(n: int, src, dst, w) -> sp.csr_matrix:
    """Weighted adjacency ``W[s, d] = sum of w_e over edges s -> d`` (Sec. 3.1)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    return sp.csr_matrix(sp.coo_matrix((w, (src, dst)), shape=(n, n)))


def adjacency_of(cfg) -> sp.csr_matrix:
    return adjacency(cfg.n, cfg.src, cfg.dst, cfg.w)


# ----------------------------------------------------------------------------- step 1-2
def attribute_similarity(a, b, omega) -> np.ndarray:
    """Cosine similarity of weighted attribute rows (Table 1, "Cos" row, in
    similarity form ``1 - distance``): ``E_ij = sum_f w_f a_if b_jf / (r_i c_j)``
    with ``r_i = sqrt(sum_f w_f a_if^2)``, ``c_j = sqrt(sum_f w_f b_jf^2)``;
    ``E_ij = 0`` where ``r_i c_j = 0``."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    w = np.asarray(omega, dtype=np.float64)
    r = np.sqrt((a * a) @ w)
    c = np.sqrt((b * b) @ w)
    num = (a * w) @ b.T
    den = np.outer(r, c)
    E = np.zeros_like(num)
    ok = den > 0
    E[ok] = num[ok] / den[ok]
    return E


def restart_term(E: np.ndarray) -> tuple[np.ndarray, float]:
    """``Ehat = E / |E|_F``; uniform ``1/sqrt(n1 n2)`` when ``|E|_F = 0``."""
    nE = float(np.sqrt(np.sum(E * E)))
    if nE > 0:
        return E / nE, nE
    return np.full(E.shape, 1.0 / np.sqrt(E.size)), 0.0


# ----------------------------------------------------------------------------- step 3
def propagate(WA: sp.csr_matrix, WB: sp.csr_matrix, X: np.ndarray) -> np.ndarray:
    """``Z = 1/2 (W_A X W_B^T + W_A^T X W_B)``.

    Entry (i, j): half the sum over successor pairs (i->u, j->v) of
    ``w_iu w_jv X_uv`` plus half the sum over predecessor pairs (u->i, v->j) of
    ``w_ui w_vj X_uv``."""
    succ = WA @ X @ WB.T
    pred = WA.T @ X @ WB
    return 0.5 * (np.asarray(succ) + np.asarray(pred))


def similarity(cfg_a, cfg_b, omega, alpha: float = 0.8, K: int = 40,
               normalize: bool = True, keep_history: bool = False) -> dict:
    """Steps 1-3: the converged similarity matrix ``X_K`` (n_a x n_b).

    Returns a dict with ``X`` (= X_K), ``Ehat``, ``nE`` (= |E|_F), ``norms``
    (``norms[k] = |Y_k|_F`` for k = 1..K, ``norms[0] = 1``), ``residual``
    (``|X_K - X_{K-1}|_F``, a diagnostic only) and, if ``keep_history``,
    ``history`` = [X_0, ..., X_K]."""
    WA = adjacency_of(cfg_a)
    WB = adjacency_of(cfg_b)
    E = attribute_similarity(cfg_a.attr, cfg_b.attr, omega)
    Ehat, nE = restart_term(E)
    X = Ehat.copy()
    hist = [X] if keep_history else None
    norms = [1.0]
    prev = X
    for _ in range(K):
        Z = propagate(WA, WB, X)
        Y = alpha * Z + (1.0 - alpha) * Ehat
        if normalize:
            nY = float(np.sqrt(np.sum(Y * Y)))
            Xn = Y / nY
        else:
            nY = 1.0
            Xn = Y
        norms.append(nY)
        prev, X = X, Xn
        if keep_history:
            hist.append(X)
    out = {"X": X, "Ehat": Ehat, "E": E, "nE": nE, "norms": np.array(norms),
           "residual": float(np.sqrt(np.sum((X - prev) ** 2)))}
    if keep_history:
        out["history"] = hist
    return out


# ----------------------------------------------------------------------------- steps 4-5
def greedy_match(X: np.ndarray) -> tuple[np.ndarray, float]:
    """Greedy matching on ``X``: visit entries by value descending, then row
    ascending, then column ascending; take an entry when its row and column
    are both still free.  Returns ``match`` (``match[i] = j`` or -1) and the
    graph score ``sum_i X[i, match[i]]`` over matched rows."""
    X = np.asarray(X, dtype=np.float64)
    n1, n2 = X.shape
    rows, cols = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    order = np.lexsort((cols.ravel(), rows.ravel(), -X.ravel()))  # last key is primary
    match = np.full(n1, -1, dtype=np.int64)
    col_used = np.zeros(n2, dtype=bool)
    need = min(n1, n2)
    taken = 0
    for flat in order:
        if taken == need:
            break
        i, j = divmod(int(flat), n2)
        if match[i] < 0 and not col_used[j]:
            match[i] = j
            col_used[j] = True
            taken += 1
    score = float(sum(X[i, match[i]] for i in range(n1) if match[i] >= 0))
    return match, score


def optimal_match(X: np.ndarray) -> tuple[np.ndarray, float]:
    """Maximum-weight assignment of ``min(n1, n2)`` pairs (the "best matching"
    alternative to step 4), via scipy's rectangular assignment solver."""
    from scipy.optimize import linear_sum_assignment

    X = np.asarray(X, dtype=np.float64)
    r, c = linear_sum_assignment(X, maximize=True)
    match = np.full(X.shape[0], -1, dtype=np.int64)
    match[r] = c
    return match, float(X[r, c].sum())


def pair_score(cfg_a, cfg_b, omega, alpha=0.8, K=40) -> tuple[np.ndarray, np.ndarray, float]:
    """Steps 1-5 for one ordered pair: ``(X_K, match, score)``."""
    X = similarity(cfg_a, cfg_b, omega, alpha, K)["X"]
    m, s = greedy_match(X)
    return X, m, s


# ----------------------------------------------------------------------------- step 6
def score_gradient(cfg_a, cfg_b, omega, alpha=0.8, K=40, gbar=1.0, match=None,
                   normalize: bool = True) -> dict:
    """Reverse mode of steps 1-5 for one pair, the matching held fixed.

    Upstream ``gbar`` multiplies ``ds``.  Returns gradients with respect to
    every user edge weight of A and of B (user edge order; duplicate edges
    share the gradient of their summed entry), and with respect to ``omega``.

    Adjoint recurrences, k = K-1 .. 0 (all products dense or sparse-dense)::

        Xbar_K   = gbar * 1[matched entries]
        Ybar     = (Xbar_{k+1} - <Xbar_{k+1}, X_{k+1}> X_{k+1}) / |Y_{k+1}|
        Ehatbar += (1 - alpha) Ybar ;  Zbar = alpha Ybar
        Wbar_A  += 1/2 (Zbar W_B X_k^T + X_k W_B Zbar^T)   at the edges of A
        Wbar_B  += 1/2 (Zbar^T W_A X_k + X_k^T W_A Zbar)   at the edges of B
        Xbar_k   = 1/2 (W_A^T Zbar W_B + W_A Zbar W_B^T)   (the operator is self-adjoint)

    then ``Ehatbar += Xbar_0``, ``Ebar = (Ehatbar - <Ehatbar, Ehat> Ehat) / |E|``
    and ``omegabar_f = sum_ij Ebar_ij dE_ij/domega_f`` with
    ``dE_ij/domega_f = a_if b_jf/(r_i c_j) - E_ij (a_if^2/(2 r_i^2) + b_jf^2/(2 c_j^2))``."""
    fw = similarity(cfg_a, cfg_b, omega, alpha, K, normalize=normalize, keep_history=True)
    hist, norms, Ehat, E, nE = fw["history"], fw["norms"], fw["Ehat"], fw["E"], fw["nE"]
    if match is None:
        match, _ = greedy_match(fw["X"])
    WA = adjacency_of(cfg_a)
    WB = adjacency_of(cfg_b)
    sa, da = np.asarray(cfg_a.src, np.int64), np.asarray(cfg_a.dst, np.int64)
    sb, db = np.asarray(cfg_b.src, np.int64), np.asarray(cfg_b.dst, np.int64)
    n1, n2 = hist[0].shape

    Xbar = np.zeros((n1, n2))
    for i in range(n1):
        if match[i] >= 0:
            Xbar[i, match[i]] = gbar
    Ehatbar = np.zeros((n1, n2))
    gA = np.zeros(sa.size)
    gB = np.zeros(sb.size)
    for k in range(K - 1, -1, -1):
        X1 = hist[k + 1]
        if normalize:
            Ybar = (Xbar - np.sum(Xbar * X1) * X1) / norms[k + 1]
        else:
            Ybar = Xbar
        Ehatbar += (1.0 - alpha) * Ybar
        Zbar = alpha * Ybar
        Xk = hist[k]
        # dZ/dW_A: (Zbar W_B X^T)[p,q] + (X W_B Zbar^T)[p,q] at each edge p->q of A
        ZWB = np.asarray(Zbar @ WB)  # (Zbar W_B)[p, j]
        XWB = np.asarray(Xk @ WB)
        gA += 0.5 * (np.einsum("ej,ej->e", ZWB[sa], Xk[da]) + np.einsum("ej,ej->e", XWB[sa], Zbar[da]))
        # dZ/dW_B: (Zbar^T W_A X)[j,v] + (X^T W_A Zbar)[j,v] at each edge j->v of B
        AX = np.asarray(WA @ Xk)
        AZ = np.asarray(WA @ Zbar)
        gB += 0.5 * (np.einsum("pe,pe->e", Zbar[:, sb], AX[:, db]) + np.einsum("pe,pe->e", Xk[:, sb], AZ[:, db]))
        Xbar = 0.5 * (np.asarray(WA.T @ Zbar @ WB) + np.asarray(WA @ Zbar @ WB.T))
    Ehatbar += Xbar

    a = np.asarray(cfg_a.attr, np.float64)
    b = np.asarray(cfg_b.attr, np.float64)
    w = np.asarray(omega, np.float64)
    gO = np.zeros(w.size)
    if nE > 0:
        Ebar = (Ehatbar - np.sum(Ehatbar * Ehat) * Ehat) / nE
        r = np.sqrt((a * a) @ w)
        c = np.sqrt((b * b) @ w)
        live = np.outer(r, c) > 0
        rs = np.where(r > 0, r, 1.0)
        cs = np.where(c > 0, c, 1.0)
        Eb = np.where(live, Ebar, 0.0)
        # term 1: sum_ij Ebar_ij a_if b_jf / (r_i c_j)
        gO += np.einsum("ij,if,jf->f", Eb / np.outer(rs, cs), a, b)
        # terms 2-3: - sum_ij Ebar_ij E_ij (a_if^2 / (2 r_i^2) + b_jf^2 / (2 c_j^2))
        EbE = Eb * E
        gO -= np.einsum("i,if->f", EbE.sum(axis=1), (a * a) / (2.0 * rs[:, None] ** 2))
        gO -= np.einsum("j,jf->f", EbE.sum(axis=0), (b * b) / (2.0 * cs[:, None] ** 2))
    return {"grad_w_a": gA, "grad_w_b": gB, "grad_omega": gO, "match": match}


# ----------------------------------------------------------------------------- batches
def run_pairs(cfgs_a, cfgs_b, pairs, omega, alpha=0.8, K=40, want_X=False):
    """Steps 1-5 for every pair ``(cfgs_a[p0], cfgs_b[p1])`` of ``pairs``, one
    after another.  Returns scores, matches and (optionally) the X matrices."""
    scores = np.zeros(len(pairs))
    matches, Xs = [], []
    for k, (ia, ib) in enumerate(pairs):
        X, m, s = pair_score(cfgs_a[int(ia)], cfgs_b[int(ib)], omega, alpha, K)
        scores[k] = s
        matches.append(m)
        if want_X:
            Xs.append(X)
    return scores, matches, Xs
