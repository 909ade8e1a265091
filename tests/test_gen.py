"""The seeded generator: structure the paper's CFGs have (Sec. 3.1) and determinism."""
import collections

import numpy as np

from gen import config1, config2, config3, config4, config5, structured_cfg


def _reachable(c):
    adj = collections.defaultdict(list)
    for s, d in zip(c.src, c.dst):
        adj[int(s)].append(int(d))
    seen, st = {0}, [0]
    while st:
        v = st.pop()
        for u in adj[v]:
            if u not in seen:
                seen.add(u)
                st.append(u)
    return len(seen)


def test_cfg_structure():
    for c in config2(40).cfgs_a + config3(3).cfgs_a:
        assert _reachable(c) == c.n  # a path from START to every block
        assert (c.src != c.n - 1).all()  # STOP has no out-edges
        sums = np.bincount(c.src, weights=c.w.astype(np.float64), minlength=c.n)
        assert np.allclose(sums[:-1], 1.0, atol=1e-6)  # right-stochastic rows
        assert len(set(zip(c.src.tolist(), c.dst.tolist()))) == c.n_edges
        assert (c.attr >= 0).all() and np.isfinite(c.attr).all()


def test_sizes_and_determinism():
    w1, w1b = config1(), config1()
    assert len(w1.pairs) == 28
    assert all(5 <= c.n <= 20 for c in w1.cfgs_a)
    for c, d in zip(w1.cfgs_a, w1b.cfgs_a):
        assert c.n == d.n and (c.src == d.src).all() and (c.w == d.w).all() and (c.attr == d.attr).all()
    w2 = config2(30)
    assert all(8 <= c.n <= 120 for c in w2.cfgs_a) and w2.F == 13
    assert all(c.attr.shape[1] == 13 for c in w2.cfgs_a)
    w4 = config4(8)
    assert len(w4.pairs) == 8 and all(10 <= c.n <= 300 for c in w4.cfgs_a)
    w5 = config5(2, 20)
    assert len(w5.pairs) == 40 and w5.F == 25 and not w5.shared


def test_exact_block_counts():
    rng = np.random.default_rng(0)
    for n in [1, 2, 3, 4, 7, 50, 333]:
        assert structured_cfg(rng, n, 5, 4).n == n
