"""Pins for the FP64 oracle, each tied to something other than the oracle itself.

The paper prints no output of the measure for a concrete input, so the pins are:
hand-derived values, a fixed point that follows from the definition, the
Kronecker linear system of Table 1 solved by ``numpy.linalg.solve``,
brute-force matching, symmetry / relabelling invariants, central finite
differences for the gradient, and the paper's Fig. 3 matrices used as inputs.
The last test plants mistakes in the oracle (on the CPU) and checks that the
pins catch each one.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import isorank
from gen import CFG, config1, structured_cfg


def cfg_from_dict(d) -> CFG:
    return CFG(n=d["n"], src=np.array(d["src"], np.int32), dst=np.array(d["dst"], np.int32),
               w=np.array(d["w"], np.float32), attr=np.array(d["attr"], np.float32))


def small_cfgs():
    return config1().cfgs_a


# ------------------------------------------------------------------ step 1: cosine term
def check_cosine_closed_form():
    a = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 0.0]])
    b = np.array([[0.0, 1.0], [3.0, 4.0]])
    E = isorank.attribute_similarity(a, b, [1.0, 1.0])
    want = np.array([[0.0, 3.0 / 5.0], [1.0 / math.sqrt(2.0), 7.0 / (5.0 * math.sqrt(2.0))], [0.0, 0.0]])
    ok1 = np.allclose(E, want, atol=1e-15)
    # weighted: omega = (4, 1): <a1,b1>_w = 4*3 = 12 for a=(1,0), b=(3,4): r = 2, c = sqrt(36+16)
    E2 = isorank.attribute_similarity(a[:1], b[1:], [4.0, 1.0])
    ok2 = abs(E2[0, 0] - 12.0 / (2.0 * math.sqrt(52.0))) < 1e-15
    return ok1 and ok2


def test_cosine_closed_form():
    assert check_cosine_closed_form()


def test_cosine_self_is_one():
    c = small_cfgs()[0]
    E = isorank.attribute_similarity(c.attr, c.attr, np.ones(13))
    assert np.allclose(np.diag(E), 1.0, atol=1e-14)
    assert (E <= 1.0 + 1e-14).all() and (E >= 0).all()


# ------------------------------------------------------------------ step 3: one iteration by hand
def check_hand_one_iteration(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hand_chain_2x3.json")))
    A, B = cfg_from_dict(g["A"]), cfg_from_dict(g["B"])
    out = isorank.similarity(A, B, g["omega"], alpha=g["alpha"], K=g["K"])
    ok_x = np.allclose(out["X"], np.array(g["X1"]), atol=1e-15)
    m, s = isorank.greedy_match(out["X"])
    return ok_x and list(m) == g["match"] and abs(s - g["score"]) < 1e-15


def test_hand_one_iteration(golden_dir):
    assert check_hand_one_iteration(golden_dir)


# ------------------------------------------------------------------ fixed point
def check_fixed_point(alpha):
    A = CFG(2, np.array([0], np.int32), np.array([1], np.int32), np.array([1.0], np.float32),
            np.array([[1.0, 0.0], [0.0, 1.0]], np.float32))
    X = isorank.similarity(A, A, [1.0, 1.0], alpha=alpha, K=40)["X"]
    m, s = isorank.greedy_match(X)
    return np.allclose(X, np.eye(2) / math.sqrt(2.0), atol=1e-15) and list(m) == [0, 1] and abs(s - math.sqrt(2.0)) < 1e-14


@pytest.mark.parametrize("alpha", [0.0, 0.5, 0.8, 0.95])
def test_fixed_point(alpha):
    # E = I, Ehat = I/sqrt2; Z(Ehat) = Ehat/2 for the 2-chain, so Y = (1 - alpha/2) Ehat
    assert check_fixed_point(alpha)


# ------------------------------------------------------------------ symmetry, equivariance, self
def check_symmetry():
    cs = small_cfgs()
    om = np.linspace(0.5, 1.5, 13)
    for (p, q) in [(0, 1), (2, 5), (3, 7)]:
        X = isorank.similarity(cs[p], cs[q], om, 0.8, 40)["X"]
        Xt = isorank.similarity(cs[q], cs[p], om, 0.8, 40)["X"]
        if not np.abs(X - Xt.T).max() <= 1e-14:
            return False
    return True


def test_symmetry():
    assert check_symmetry()


def permute_cfg(c: CFG, perm: np.ndarray) -> CFG:
    """Relabel block i as perm[i]."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    attr = c.attr[inv]
    return CFG(c.n, perm[c.src].astype(np.int32), perm[c.dst].astype(np.int32), c.w.copy(), attr)


def test_relabelling_equivariance():
    cs = small_cfgs()
    A, B = cs[1], cs[4]
    om = np.ones(13)
    X = isorank.similarity(A, B, om, 0.8, 40)["X"]
    m, s = isorank.greedy_match(X)
    rng = np.random.default_rng(7)
    perm = rng.permutation(A.n)
    Xp = isorank.similarity(permute_cfg(A, perm), B, om, 0.8, 40)["X"]
    # row perm[i] of Xp is row i of X
    assert np.abs(Xp[perm] - X).max() <= 1e-14
    mp, sp_ = isorank.greedy_match(Xp)
    assert abs(sp_ - s) <= 1e-13
    assert all(mp[perm[i]] == m[i] for i in range(A.n))


def test_self_similarity():
    c = small_cfgs()[2]
    om = np.ones(13)
    X = isorank.similarity(c, c, om, 0.8, 40)["X"]
    assert np.abs(X - X.T).max() <= 1e-14
    # alpha = 0: X = E/|E|, identity matching, s = n/|E|_F
    E = isorank.attribute_similarity(c.attr, c.attr, om)
    X0 = isorank.similarity(c, c, om, 0.0, 40)["X"]
    assert np.allclose(X0, E / np.linalg.norm(E), atol=1e-15)
    m, s = isorank.greedy_match(X0)
    assert list(m) == list(range(c.n))
    assert abs(s - c.n / np.linalg.norm(E)) < 1e-13


# ------------------------------------------------------------------ Table 1 linear system
def check_linear_system(A: CFG, B: CFG, alpha: float, om) -> float:
    WA = isorank.adjacency_of(A).toarray()
    WB = isorank.adjacency_of(B).toarray()
    # column-major vec: vec(W_A X W_B^T) = (W_B kron W_A) vec X
    M = 0.5 * (np.kron(WB, WA) + np.kron(WB.T, WA.T))
    E = isorank.attribute_similarity(A.attr, B.attr, om)
    e = (E / np.linalg.norm(E)).ravel(order="F")
    x = np.linalg.solve(np.eye(M.shape[0]) - alpha * M, (1.0 - alpha) * e)
    X = isorank.similarity(A, B, om, alpha=alpha, K=2000, normalize=False)["X"]
    return float(np.abs(X.ravel(order="F") - x).max())


@pytest.mark.parametrize("alpha", [0.5, 0.8, 0.95])
def test_linear_system_limit(alpha):
    rng = np.random.default_rng(11)
    A = structured_cfg(rng, 5, 3, 3)
    B = structured_cfg(rng, 6, 3, 3)
    om = np.array([1.0, 0.5, 2.0, 1.0])
    assert check_linear_system(A, B, alpha, om) < 1e-12
    assert check_linear_system(A, A, alpha, om) < 1e-12


# ------------------------------------------------------------------ matching
def naive_greedy(X):
    """Sequential greedy by repeated global argmax (a second algorithm for the
    same definition: largest value, then smaller row, then smaller column)."""
    X = np.array(X, dtype=np.float64)
    n1, n2 = X.shape
    alive_r, alive_c = set(range(n1)), set(range(n2))
    m = [-1] * n1
    while alive_r and alive_c:
        best = None
        for i in sorted(alive_r):
            for j in sorted(alive_c):
                if best is None or X[i, j] > X[best]:
                    best = (i, j)
        m[best[0]] = best[1]
        alive_r.discard(best[0])
        alive_c.discard(best[1])
    return m


def brute_best(X):
    n1, n2 = X.shape
    best = -1.0
    if n1 <= n2:
        for cols in itertools.permutations(range(n2), n1):
            best = max(best, sum(X[i, cols[i]] for i in range(n1)))
    else:
        for rows in itertools.permutations(range(n1), n2):
            best = max(best, sum(X[rows[j], j] for j in range(n2)))
    return best


def test_greedy_equals_sequential_and_brute_force_bounds():
    rng = np.random.default_rng(3)
    for trial in range(60):
        n1, n2 = int(rng.integers(1, 8)), int(rng.integers(1, 8))
        X = rng.random((n1, n2))
        if trial % 3 == 0:  # ties: quantised values
            X = np.round(X * 4) / 4
        m, s = isorank.greedy_match(X)
        assert list(m) == naive_greedy(X)
        assert sum(1 for v in m if v >= 0) == min(n1, n2)
        assert len(set(v for v in m if v >= 0)) == min(n1, n2)
        opt = brute_best(X)
        mo, so = isorank.optimal_match(X)
        assert abs(so - opt) < 1e-12
        assert s >= 0.5 * opt - 1e-12


# ------------------------------------------------------------------ gradient vs finite differences
def _score_fixed_match(A, B, om, alpha, K, match):
    X = isorank.similarity(A, B, om, alpha, K)["X"]
    return sum(X[i, match[i]] for i in range(A.n) if match[i] >= 0)


def greedy_margin(X):
    """Smallest gap between a greedy pick and the best competitor in its row or column."""
    m, _ = isorank.greedy_match(X)
    X = np.array(X)
    n1, n2 = X.shape
    order = sorted([(X[i, m[i]], i, m[i]) for i in range(n1) if m[i] >= 0], key=lambda t: (-t[0], t[1]))
    alive_r, alive_c = set(range(n1)), set(range(n2))
    gap = np.inf
    for v, i, j in order:
        comp = [X[i, c] for c in alive_c if c != j] + [X[r, j] for r in alive_r if r != i]
        if comp:
            gap = min(gap, v - max(comp))
        alive_r.discard(i)
        alive_c.discard(j)
    return gap


def check_gradient_fd(A, B, om, alpha=0.8, K=40, h=1e-6, tol=1e-7):
    X = isorank.similarity(A, B, om, alpha, K)["X"]
    m, _ = isorank.greedy_match(X)
    g = isorank.score_gradient(A, B, om, alpha, K, gbar=1.0, match=m)
    worst = 0.0
    for side, cfg, key in (("a", A, "grad_w_a"), ("b", B, "grad_w_b")):
        for e in range(cfg.n_edges):
            wp = cfg.w.astype(np.float64).copy()
            wm = wp.copy()
            wp[e] += h
            wm[e] -= h
            Cp = CFG(cfg.n, cfg.src, cfg.dst, wp, cfg.attr)
            Cm = CFG(cfg.n, cfg.src, cfg.dst, wm, cfg.attr)
            if side == "a":
                fd = (_score_fixed_match(Cp, B, om, alpha, K, m) - _score_fixed_match(Cm, B, om, alpha, K, m)) / (2 * h)
            else:
                fd = (_score_fixed_match(A, Cp, om, alpha, K, m) - _score_fixed_match(A, Cm, om, alpha, K, m)) / (2 * h)
            worst = max(worst, abs(fd - g[key][e]) / max(1.0, abs(fd)))
    for f in range(len(om)):
        op = np.array(om, np.float64)
        omn = op.copy()
        op[f] += h
        omn[f] -= h
        fd = (_score_fixed_match(A, B, op, alpha, K, m) - _score_fixed_match(A, B, omn, alpha, K, m)) / (2 * h)
        worst = max(worst, abs(fd - g["grad_omega"][f]) / max(1.0, abs(fd)))
    return worst <= tol, worst


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    done = 0
    for _ in range(20):
        A = structured_cfg(rng, int(rng.integers(5, 11)), 3, 4)
        B = structured_cfg(rng, int(rng.integers(5, 11)), 3, 4)
        om = rng.uniform(0.5, 1.5, 5)
        if greedy_margin(isorank.similarity(A, B, om)["X"]) < 1e-3:
            continue
        ok, worst = check_gradient_fd(A, B, om)
        assert ok, worst
        done += 1
        if done == 3:
            break
    assert done >= 2


def test_gradient_linear_mode_matches_finite_differences():
    rng = np.random.default_rng(9)
    A = structured_cfg(rng, 6, 3, 3)
    B = structured_cfg(rng, 7, 3, 3)
    om = np.array([1.0, 0.7, 1.3, 0.9])
    X = isorank.similarity(A, B, om, 0.6, 12, normalize=False)["X"]
    m, _ = isorank.greedy_match(X)
    g = isorank.score_gradient(A, B, om, 0.6, 12, 1.0, m, normalize=False)
    h = 1e-6
    wp, wm = A.w.astype(np.float64).copy(), A.w.astype(np.float64).copy()
    wp[0] += h
    wm[0] -= h

    def sc(Acfg):
        Xs = isorank.similarity(Acfg, B, om, 0.6, 12, normalize=False)["X"]
        return sum(Xs[i, m[i]] for i in range(A.n) if m[i] >= 0)

    fd = (sc(CFG(A.n, A.src, A.dst, wp, A.attr)) - sc(CFG(A.n, A.src, A.dst, wm, A.attr))) / (2 * h)
    assert abs(fd - g["grad_w_a"][0]) <= 1e-7 * max(1.0, abs(fd))


# ------------------------------------------------------------------ degenerate inputs
def test_zero_attributes_give_uniform_restart():
    A = CFG(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.ones(2, np.float32), np.zeros((3, 2), np.float32))
    B = CFG(2, np.array([0], np.int32), np.array([1], np.int32), np.ones(1, np.float32), np.zeros((2, 2), np.float32))
    out = isorank.similarity(A, B, [1.0, 1.0], 0.8, 0)
    assert np.allclose(out["X"], 1.0 / math.sqrt(6.0), atol=1e-15)
    g = isorank.score_gradient(A, B, [1.0, 1.0], 0.8, 5)
    assert np.all(g["grad_omega"] == 0)


def test_single_block_and_no_edges():
    A = CFG(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32), np.ones((1, 3), np.float32))
    B = CFG(4, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
            np.array([[1, 0, 0], [1, 1, 1], [0, 0, 2], [0, 0, 0]], np.float32))
    X = isorank.similarity(A, B, np.ones(3), 0.8, 40)["X"]
    # no edges: Z = 0, Y = (1-alpha) Ehat, X = Ehat at every step
    E = isorank.attribute_similarity(A.attr, B.attr, np.ones(3))
    assert np.allclose(X, E / np.linalg.norm(E), atol=1e-15)
    m, s = isorank.greedy_match(X)
    assert list(m) == [1] and abs(s - X[0, 1]) < 1e-15


# ------------------------------------------------------------------ Fig. 3 input fixture
def fig3_cfgs(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fig3_pathfinder.json")))
    out = []
    for key in ("kepler", "maxwell"):
        M = np.array(g[key]["matrix"])
        n = M.shape[0]
        off = M - np.diag(np.diag(M))
        s, d = np.nonzero(off)
        out.append(CFG(n, s.astype(np.int32), d.astype(np.int32), off[s, d].astype(np.float32),
                       np.diag(M).reshape(n, 1).astype(np.float32)))
    return out


def test_fig3_fixture_invariants(golden_dir):
    kep, max_ = fig3_cfgs(golden_dir)
    assert kep.n == 6 and max_.n == 4
    # entries are normalised over all observations (Fig. 3 caption / Sec. 3.1)
    tot_k = kep.w.sum() + kep.attr.sum()
    tot_m = max_.w.sum() + max_.attr.sum()
    assert abs(tot_k - 0.98) < 1e-6 and abs(tot_m - 1.02) < 1e-6
    om = np.ones(1)
    X = isorank.similarity(kep, max_, om)["X"]
    Xt = isorank.similarity(max_, kep, om)["X"]
    assert np.abs(X - Xt.T).max() <= 1e-14
    assert abs(np.linalg.norm(X) - 1.0) < 1e-14
    m, s = isorank.greedy_match(X)
    assert sum(1 for v in m if v >= 0) == 4
    assert 0 < s <= math.sqrt(4) + 1e-12


# ------------------------------------------------------------------ planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch, golden_dir):
    """Each plausible slip in the iteration must break at least one pin."""
    real = isorank.propagate

    def drop_pred(WA, WB, X):
        return 0.5 * np.asarray(WA @ X @ WB.T)

    def transposed_b(WA, WB, X):
        return 0.5 * (np.asarray(WA @ X @ WB) + np.asarray(WA.T @ X @ WB.T))

    def no_half(WA, WB, X):
        return 2.0 * real(WA, WB, X)

    def succ_twice(WA, WB, X):
        return np.asarray(WA @ X @ WB.T)

    rng = np.random.default_rng(11)
    A = structured_cfg(rng, 5, 3, 3)
    B = structured_cfg(rng, 6, 3, 3)
    om = np.array([1.0, 0.5, 2.0, 1.0])
    for bad in (drop_pred, transposed_b, no_half, succ_twice):
        monkeypatch.setattr(isorank, "propagate", bad)
        caught = (not check_hand_one_iteration(golden_dir)) or check_linear_system(A, B, 0.8, om) > 1e-9
        monkeypatch.setattr(isorank, "propagate", real)
        assert caught, bad.__name__

    # a wrong cosine normaliser
    real_att = isorank.attribute_similarity

    def wrong_cos(a, b, omega):
        return real_att(a, b, np.sqrt(np.asarray(omega, np.float64)))

    monkeypatch.setattr(isorank, "attribute_similarity", wrong_cos)
    assert not check_cosine_closed_form()
    monkeypatch.setattr(isorank, "attribute_similarity", real_att)

    # a greedy that breaks ties by the larger index
    real_g = isorank.greedy_match

    def bad_tie(X):
        m, s = real_g(np.asarray(X)[::-1, ::-1])
        n1, n2 = np.asarray(X).shape
        out = np.full(n1, -1)
        for i in range(n1):
            if m[i] >= 0:
                out[n1 - 1 - i] = n2 - 1 - m[i]
        return out, s

    monkeypatch.setattr(isorank, "greedy_match", bad_tie)
    assert not check_hand_one_iteration(golden_dir)
    monkeypatch.setattr(isorank, "greedy_match", real_g)


def test_query_pruning_bound_holds_and_is_tight():
    """The bound a query search could prune with: s <= sqrt(min(n_a, n_b)),
    the Cauchy-Schwarz bound on a sum of min(n_a, n_b) entries of a
    nonnegative X with |X|_F = 1.  It holds on every pair of the parity and
    query workloads' distributions, for every alpha; and no smaller bound in
    sizes alone exists, since X = I / sqrt(n) (two identical chains with
    one-hot attributes at alpha = 0) reaches it exactly."""
    from gen import config1, config5

    for w in (config1(), config5(2, 12)):
        for alpha in (0.0, 0.5, 0.8, 0.95):
            for a, b in w.pairs:
                A, B = w.cfgs_a[a], w.cfgs_b[b]
                X = oracle.similarity(A, B, np.ones(w.F), alpha, 40)["X"]
                assert abs(np.linalg.norm(X) - 1.0) < 1e-12 and X.min() >= 0.0
                s = oracle.greedy_match(X)[1]
                assert s <= np.sqrt(min(A.n, B.n)) + 1e-12
    # tightness: n blocks, no edges, attributes one-hot per block
    n = 5
    cfg = CFG(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
              np.eye(n, dtype=np.float32))
    X = oracle.similarity(cfg, cfg, np.ones(n), 0.0, 40)["X"]
    assert abs(oracle.greedy_match(X)[1] - np.sqrt(n)) < 1e-12
