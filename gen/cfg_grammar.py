"""Seeded synthetic control-flow graphs shaped like GPU-kernel CFGs.

This module only draws random structure and random block attributes.  It holds
no part of the similarity arithmetic, so both the FP64 oracle and the CUDA path
can consume its output without sharing any of the method's code.

Shape of the graphs (paper Sec. 3.1, "Kernel Control Flow Graphs", and the
CFG drawings of Fig. 2): a unique START block with a path to every block, a
unique STOP block, basic blocks as nodes and jumps as directed edges.  Bodies
are nested sequence / if-then-else diamond / while-loop regions, the shapes a
structured kernel compiles to.  Loops carry a back edge, so graphs have cycles
even though the paper calls a CFG a DAG.  A few blocks get an early-return
edge to STOP or a break edge to their loop's exit, which gives STOP and loop
exits in-degrees above two, as guard clauses (``if (tid >= n) return;``) do.

Attributes per block (paper Sec. 1 and 3.1: instruction-operation mix,
registers allocated, block execution frequency): ``n_cat`` instruction-category
counts ~ Poisson(lambda), lambda ~ U[0, 20] drawn per (block, category), then
one extra column: a register count ~ U{8..64} or a block execution frequency
~ lognormal(0, 2).  Edge weights are branch probabilities: the out-edges of a
block get a Dirichlet(1, ..., 1) draw (paper Sec. 3.1, "Transition
probability": each row of the transition matrix sums to one); STOP has none.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CFG:
    """One control-flow graph: ``n`` blocks, edges ``src[e] -> dst[e]`` with
    weight ``w[e]`` and a row-major attribute matrix ``attr`` of shape [n, F]."""

    n: int
    src: np.ndarray  # int32 [E]
    dst: np.ndarray  # int32 [E]
    w: np.ndarray  # float32 [E]
    attr: np.ndarray  # float32 [n, F]

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])


class _Builder:
    """Budgeted recursive region grammar: every call creates exactly the number
    of blocks it is given, so a CFG with an exact block count is drawn in one
    pass (no rejection loop)."""

    def __init__(self, rng: np.random.Generator, unroll: bool, p_ret: float, p_brk: float):
        self.rng = rng
        self.unroll = unroll
        self.p_ret = p_ret
        self.p_brk = p_brk
        self.n = 0
        self.edges: list[tuple[int, int]] = []
        self.loop_exits: list[int] = []  # pending (filled lazily) exit ids of enclosing loops
        self.plain_blocks: list[tuple[int, int]] = []  # (block, innermost loop exit or -1)

    def new(self) -> int:
        v = self.n
        self.n += 1
        return v

    def chain(self, k: int) -> tuple[int, int]:
        first = prev = self.new()
        self.plain_blocks.append((first, self.loop_exits[-1] if self.loop_exits else -1))
        for _ in range(k - 1):
            v = self.new()
            self.plain_blocks.append((v, self.loop_exits[-1] if self.loop_exits else -1))
            self.edges.append((prev, v))
            prev = v
        return first, prev

    def region(self, budget: int, depth: int) -> tuple[int, int]:
        assert budget >= 1
        if depth <= 0 or budget < 3:
            return self.chain(budget)
        kind = self.rng.choice(3, p=[0.40, 0.35, 0.25])
        if kind == 0:  # sequence of 2..4 sub-regions
            k = int(self.rng.integers(2, min(4, budget) + 1))
            cuts = np.sort(self.rng.choice(np.arange(1, budget), size=k - 1, replace=False))
            sizes = np.diff(np.concatenate([[0], cuts, [budget]])).tolist()
            entry = exit_ = None
            for s in sizes:
                e0, e1 = self.region(int(s), depth - 1)
                if entry is None:
                    entry = e0
                else:
                    self.edges.append((exit_, e0))
                exit_ = e1
            return entry, exit_
        if kind == 1:  # if-then[-else] diamond: cond, then, [else], join
            cond = self.new()
            inner = budget - 2
            with_else = inner >= 2 and self.rng.random() < 0.6
            b1 = int(self.rng.integers(1, inner)) if with_else else inner
            t0, t1 = self.region(b1, depth - 1)
            if with_else:
                f0, f1 = self.region(inner - b1, depth - 1)
            join = self.new()
            self.edges.append((cond, t0))
            self.edges.append((t1, join))
            if with_else:
                self.edges.append((cond, f0))
                self.edges.append((f1, join))
            else:
                self.edges.append((cond, join))
            return cond, join
        # while loop: header, body (optionally unrolled u times), exit
        header = self.new()
        inner = budget - 2
        u = int(self.rng.integers(4, 17)) if self.unroll else 1
        if u > 1 and inner // u >= 1:
            body = inner // u
            extra = inner - u * body  # leftover blocks become a chain before the exit
        else:
            u, body, extra = 1, inner, 0
        exit_placeholder = -(len(self.loop_exits) + 2)  # resolved once the exit exists
        self.loop_exits.append(exit_placeholder)
        if u == 1:
            b_first, b_last = self.region(body, depth - 1)
        else:
            # one body template, instantiated u times back to back
            tmpl = _Builder(self.rng, False, 0.0, 0.0)
            t_entry, t_exit = tmpl.region(body, depth - 1)
            b_first = prev_exit = None
            for _ in range(u):
                off = self.n
                for _ in range(tmpl.n):
                    self.plain_blocks.append((self.new(), exit_placeholder))
                for (a, c) in tmpl.edges:
                    self.edges.append((a + off, c + off))
                if prev_exit is None:
                    b_first = off + t_entry
                else:
                    self.edges.append((prev_exit, off + t_entry))
                prev_exit = off + t_exit
            b_last = prev_exit
        self.loop_exits.pop()
        if extra > 0:
            c0, c1 = self.chain(extra)
            self.edges.append((header, b_first))
            self.edges.append((b_last, header))
            self.edges.append((header, c0))
            tail = c1
        else:
            self.edges.append((header, b_first))
            self.edges.append((b_last, header))
            tail = None
        exit_ = self.new()
        if tail is None:
            self.edges.append((header, exit_))
        else:
            self.edges.append((tail, exit_))
        # resolve break targets of this loop
        self.plain_blocks = [(v, exit_ if t == exit_placeholder else t) for (v, t) in self.plain_blocks]
        return header, exit_


def structured_cfg(
    rng: np.random.Generator,
    n: int,
    depth_max: int,
    n_cat: int,
    extra: str = "registers",
    unroll: bool = False,
    p_ret: float = 0.03,
    p_brk: float = 0.05,
) -> CFG:
    """Draw one CFG with exactly ``n`` blocks (``n >= 1``).

    Block 0 is START and block n-1 is STOP (paper Sec. 3.1).  ``extra`` picks the
    last attribute column: ``"registers"`` (U{8..64}) or ``"freq"``
    (lognormal(0, 2) block execution frequency)."""
    if n < 1:
        raise ValueError("a CFG has at least one block")
    b = _Builder(rng, unroll, p_ret, p_brk)
    if n == 1:
        b.new()
    elif n == 2:
        s, t = b.new(), b.new()
        b.edges.append((s, t))
    else:
        start = b.new()
        r0, r1 = b.region(n - 2, depth_max)
        stop = b.new()
        b.edges.append((start, r0))
        b.edges.append((r1, stop))
        # early returns and loop breaks (guard clauses); never from START/STOP
        for (v, brk) in b.plain_blocks:
            if rng.random() < p_ret:
                b.edges.append((v, stop))
            elif brk >= 0 and rng.random() < p_brk:
                b.edges.append((v, brk))
    assert b.n == n, (b.n, n)
    edges = sorted(set(b.edges))
    src = np.array([e[0] for e in edges], dtype=np.int32)
    dst = np.array([e[1] for e in edges], dtype=np.int32)
    # Dirichlet(1,...,1) branch probabilities per block over its out-edges
    w = np.zeros(len(edges), dtype=np.float64)
    for v in range(n):
        idx = np.flatnonzero(src == v)
        if idx.size:
            w[idx] = rng.dirichlet(np.ones(idx.size))
    # attributes: n_cat Poisson counts with per-(block, category) rates, + 1 extra
    lam = rng.uniform(0.0, 20.0, size=(n, n_cat))
    cats = rng.poisson(lam).astype(np.float64)
    if extra == "registers":
        last = rng.integers(8, 65, size=(n, 1)).astype(np.float64)
    elif extra == "freq":
        last = rng.lognormal(0.0, 2.0, size=(n, 1))
    else:
        raise ValueError(extra)
    attr = np.concatenate([cats, last], axis=1).astype(np.float32)
    return CFG(n=n, src=src, dst=dst, w=w.astype(np.float32), attr=attr)


def loguniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    """Integer drawn log-uniformly from [lo, hi]."""
    v = int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1)))))
    return min(max(v, lo), hi)
