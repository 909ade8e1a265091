"""The path on several GPUs, one process per GPU.

Pairs are independent, so the path shards by pairs: every rank holds the
whole pack (a few MB to about 60 MB) and computes its part of the pair
list.  The exchange steps:

- scores: an all-gather of every rank's scores back into pair order;
- the query workload: every rank's top-k candidates of each query (from its
  part of the corpus) are all-gathered and merged per query, ties going to
  the smaller corpus index as in the one-GPU top-k;
- gradients: an all-reduce (sum) of the omega gradient and of the edge
  gradients, which every rank accumulates from its own pairs into
  full-length buffers.

The partition is LPT (longest processing time first): pairs in descending
order of the plan's cost measure n_a n_b + 2 e_a e_b (ties: smaller pair
index first), each to the rank with the least total cost so far (ties: the
smaller rank).  torch.distributed carries the collectives (NCCL on GPUs,
gloo on CPU ranks in tests).
"""
from __future__ import annotations

import heapq

import numpy as np


def pair_costs(n_a, n_b, e_a, e_b, pairs) -> np.ndarray:
    """Per-pair cost n_a n_b + 2 e_a e_b (blocks and distinct edges per CFG of
    each side, pairs [P, 2])."""
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    a, b = pairs[:, 0], pairs[:, 1]
    n_a, n_b = np.asarray(n_a, np.int64), np.asarray(n_b, np.int64)
    e_a, e_b = np.asarray(e_a, np.int64), np.asarray(e_b, np.int64)
    return n_a[a] * n_b[b] + 2 * e_a[a] * e_b[b]


def lpt_partition(costs, world: int) -> list[np.ndarray]:
    """Pair indices of every rank (ascending), by LPT on `costs`."""
    costs = np.asarray(costs, np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.lexsort((np.arange(len(costs)), -costs))
    owner = np.empty(len(costs), np.int64)
    heap = [(0, r) for r in range(world)]
    for p in order:
        load, r = heapq.heappop(heap)
        owner[p] = r
        heapq.heappush(heap, (load + int(costs[p]), r))
    return [np.flatnonzero(owner == r) for r in range(world)]


class ScoreGather:
    """All-gather of every rank's scores back into pair order, for a fixed
    partition (every rank derives the same one, so no sizes are exchanged and
    nothing waits on the host): ``gather(local_scores) -> scores of all P
    pairs`` on every rank."""

    def __init__(self, parts, P: int, device, dtype=None, group=None):
        import torch

        self.group = group
        self.counts = [len(p) for p in parts]
        self.m = max(max(self.counts), 1)
        self.dtype = dtype or torch.float32
        self.idx = [torch.as_tensor(np.asarray(p, np.int64), device=device) for p in parts]
        self.pad = torch.zeros(self.m, dtype=self.dtype, device=device)
        self.bufs = [torch.zeros(self.m, dtype=self.dtype, device=device) for _ in parts]
        self.full = torch.zeros(P, dtype=self.dtype, device=device)

    def __call__(self, local_scores):
        import torch.distributed as dist

        n = local_scores.shape[0]
        self.pad[:n] = local_scores
        dist.all_gather(self.bufs, self.pad, group=self.group)
        for r, (i, c) in enumerate(zip(self.idx, self.counts)):
            self.full[i] = self.bufs[r][:c]
        return self.full


def merge_topk(local_top, local_ids, k: int, group=None, select=None):
    """The global top-k of each query from every rank's local top-k.

    local_top [Q, k] float32 and local_ids [Q, k] int64 (global corpus
    indices; a rank with fewer than k corpus entries pads with -inf and -1).
    select(scores [Q, C], ids [Q, C], k) -> (top [Q, k], ids [Q, k]) picks the
    k largest per row, ties to the smaller id; by default the library's
    cf_topk on the device, applied to the candidates ordered by corpus index
    so that its ties-to-the-smaller-column rule is ties-to-the-smaller-index."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    lt = local_top.contiguous()
    li = local_ids.to(torch.int64).contiguous()
    tops = [torch.empty_like(lt) for _ in range(world)]
    ids = [torch.empty_like(li) for _ in range(world)]
    dist.all_gather(tops, lt, group=group)
    dist.all_gather(ids, li, group=group)
    cand_s = torch.cat(tops, dim=1)  # [Q, world k], rank by rank
    cand_i = torch.cat(ids, dim=1)
    sel = select or _select_cf_topk
    return sel(cand_s, cand_i, k)


def _select_cf_topk(scores, ids, k):
    import torch

    from . import api

    order = torch.argsort(torch.where(ids < 0, torch.iinfo(torch.int64).max, ids), dim=1, stable=True)
    s_sorted = torch.gather(scores, 1, order).contiguous()
    i_sorted = torch.gather(ids, 1, order)
    top, pos = api.topk(s_sorted, k)
    return top, torch.gather(i_sorted, 1, pos.to(torch.int64))


def allreduce_sum(*tensors, group=None):
    """In-place sum over the ranks of every tensor (the gradients)."""
    import torch.distributed as dist

    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors
