"""The five seeded synthetic workloads and their pair lists.

Every CFG ``i`` of workload ``c`` is drawn from ``numpy.random.default_rng([c, i])``
(query/corpus workloads use ``[c, side, i]``), so any subset can be regenerated
on its own.  Pair lists are deterministic.  ``scale`` shrinks a workload for
fast tests without changing how its members are drawn.

| id | workload                                   | CFGs                 | pairs            | F  |
|----|--------------------------------------------|----------------------|------------------|----|
| 1  | parity: 8 CFGs, n ~ U{5..20}, depth <= 3   | 8                    | all 28 (i<j)     | 13 |
| 2  | batched: n log-uniform [8,120], depth <= 5 | 200                  | all 19,900       | 13 |
| 3  | large: n ~ U{500..2000}, depth <= 8, loops unrolled 4-16x, extra = block frequency | 64 | all 2,016 | 13 |
| 4  | gradient: n log-uniform [10,300]           | 512 (pairs 2p,2p+1)  | 256              | 13 |
| 5  | query: 32 queries x 10,000 corpus, n log-uniform [5,400], 24 categories | 32 + 10,000 | 320,000 | 25 |
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .cfg_grammar import CFG, loguniform_int, structured_cfg


@dataclass
class Workload:
    name: str
    cfgs_a: list[CFG]
    cfgs_b: list[CFG]  # the same list object as cfgs_a when both sides share one corpus
    pairs: np.ndarray  # int32 [P, 2]: (index into cfgs_a, index into cfgs_b)
    F: int
    meta: dict = field(default_factory=dict)

    @property
    def shared(self) -> bool:
        return self.cfgs_a is self.cfgs_b


def all_pairs(n: int) -> np.ndarray:
    """All unordered pairs i < j of n items, row-major."""
    i, j = np.triu_indices(n, k=1)
    return np.stack([i, j], axis=1).astype(np.int32)


def _cfgs(seed_prefix, count, draw_n, **kw) -> list[CFG]:
    out = []
    for i in range(count):
        rng = np.random.default_rng(list(seed_prefix) + [i])
        n = draw_n(rng)
        out.append(structured_cfg(rng, n, **kw))
    return out


def config1(count: int = 8) -> Workload:
    cfgs = _cfgs([1], count, lambda r: int(r.integers(5, 21)), depth_max=3, n_cat=12)
    return Workload("cfg1_parity_8cfgs_n5-20", cfgs, cfgs, all_pairs(count), 13)


def config2(count: int = 200) -> Workload:
    cfgs = _cfgs([2], count, lambda r: loguniform_int(r, 8, 120), depth_max=5, n_cat=12)
    return Workload(f"cfg2_batched_{count}cfgs_n8-120", cfgs, cfgs, all_pairs(count), 13)


def config3(count: int = 64, n_lo: int = 500, n_hi: int = 2000) -> Workload:
    cfgs = _cfgs([3], count, lambda r: int(r.integers(n_lo, n_hi + 1)), depth_max=8,
                 n_cat=12, extra="freq", unroll=True)
    return Workload(f"cfg3_large_{count}cfgs_n{n_lo}-{n_hi}", cfgs, cfgs, all_pairs(count), 13)


def config4(n_pairs: int = 256) -> Workload:
    cfgs = _cfgs([4], 2 * n_pairs, lambda r: loguniform_int(r, 10, 300), depth_max=5, n_cat=12)
    pairs = np.stack([np.arange(0, 2 * n_pairs, 2), np.arange(1, 2 * n_pairs, 2)], axis=1)
    return Workload(f"cfg4_grad_{n_pairs}pairs_n10-300", cfgs, cfgs, pairs.astype(np.int32), 13)


def config5(n_query: int = 32, n_corpus: int = 10000) -> Workload:
    draw = lambda r: loguniform_int(r, 5, 400)  # noqa: E731
    q = _cfgs([5, 0], n_query, draw, depth_max=5, n_cat=24)
    c = _cfgs([5, 1], n_corpus, draw, depth_max=5, n_cat=24)
    qi, ci = np.meshgrid(np.arange(n_query), np.arange(n_corpus), indexing="ij")
    pairs = np.stack([qi.ravel(), ci.ravel()], axis=1).astype(np.int32)
    return Workload(f"cfg5_query_{n_query}x{n_corpus}_n5-400", q, c, pairs, 25,
                    meta={"n_query": n_query, "n_corpus": n_corpus, "top_k": 16})


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}
