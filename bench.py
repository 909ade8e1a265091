#!/usr/bin/env python
"""Throughput of the batched CFG-pair similarity on one GB300 (or N, one rank each).

Workload: all 19,900 pairs of 200 seeded synthetic CFGs (block counts
log-uniform in 8..120, structured sequence / diamond / loop grammar, 12
instruction-category counts + registers per block, Dirichlet branch
probabilities), K = 40, alpha = 0.8.  One step = the whole forward hot path
over the batch: device-side plan (cost order, offsets), the persistent
iteration kernel (attribute term, 40 renormalised iterations, greedy
matching, graph score) -- through the C ABI.

Output: one JSON line on rank 0 (see the keys below).  ``--impl reference``
times the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")  # each oracle process runs one thread (cores = processes)

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import re  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CFG-pair similarity evals/sec (fwd, fwd+bwd) batched vs per-pair, % roofline"
UNIT = "pairs/s"
ALPHA, K_ITERS = 0.8, 40
WORKLOADS = {
    "cfg2": "cfg2: all 19,900 pairs of 200 seeded CFGs, n log-uniform 8-120, depth<=5, F=13 "
            "(12 instruction categories + registers), K=40, alpha=0.8, greedy matching + score",
    "cfg3": "cfg3: all 2,016 pairs of 64 seeded CFGs, n 500-2000, loops unrolled 4-16x, F=13 "
            "(12 categories + block frequency), K=40, greedy matching + score",
    "cfg4": "cfg4: 256 seeded pairs, n log-uniform 10-300, F=13, K=40: forward (scores + matchings) "
            "and the adjoint (edge-weight and omega gradients, sqrt(K) checkpoints)",
    "cfg5": "cfg5: 32 query CFGs x 10,000-CFG corpus (320,000 pairs), n log-uniform 5-400, F=25, K=40: "
            "scores, top-16 per query, then matchings of the 512 winners",
    "dist": "Table 1 distances (Euclidean, Manhattan, Minkowski p=3, Jaccard, Cosine) of the bilinearly resized "
            "transition matrices, min-max scaled to [0,1], for all 19,900 pairs of the 200 cfg2 CFGs",
    "optimal": "cfg2 forward (all 19,900 pairs, K=40) with the maximum-weight assignment instead of the greedy "
               "matching (X_K kept in HBM, one warp per pair)",
    "ward": "Ward clustering of the 200 cfg2 CFGs: the 200 x 200 score matrix from the 19,900 pair scores, then "
            "the Ward linkage of its rows (199 merges)",
}
# units of the per-workload lines (the headline and the other workloads: pairs/s)
UNITS = {"ward": "linkages/s"}
WORKLOAD = WORKLOADS["cfg2"]


# --pairs: the large-CFG workload cut to its first N pairs (a smaller case of
# the same kernel, for an ncu capture that ends in minutes); 0 = all.
PAIR_LIMIT = 0


def workload(name="cfg2"):
    import dataclasses

    from gen import config2, config3, config4, config5

    w = {"cfg2": config2, "cfg3": config3, "cfg4": config4, "cfg5": config5, "dist": config2,
         "optimal": config2, "ward": config2}[name]()
    if name == "cfg3" and PAIR_LIMIT:
        w = dataclasses.replace(w, pairs=w.pairs[:PAIR_LIMIT])
    return w


def algorithmic(w, K):
    """Per-launch algorithmic counts of the iteration kernel.

    On-chip bytes: every iteration reads each gathered neighbour-pair entry
    once (e_a * e_b successor pairs + e_a * e_b predecessor pairs), reads
    (1 - alpha) Ehat once and writes Y once per entry, 4 bytes each.
    HBM bytes: the pack (read once), the pair list, scores and matchings.
    FLOPs: attribute term n_a n_b (2F + 3) plus per iteration 4 per gathered
    pair and 5 per entry."""
    na, ea = _sizes(w.cfgs_a)
    nb, eb = _sizes(w.cfgs_b)
    a, b = w.pairs[:, 0], w.pairs[:, 1]
    nn = na[a] * nb[b]
    ee = ea[a] * eb[b]
    onchip = int((K * 4 * (2 * ee + 2 * nn)).sum())
    flops = int((nn * (2 * w.F + 3) + K * (4 * ee + 5 * nn)).sum())
    return onchip, flops, int(nn.sum()), int(na[a].sum())


def _sizes(cfgs):
    """Blocks and distinct edges of every CFG (int64 arrays)."""
    n = np.array([c.n for c in cfgs], np.int64)
    e = np.array([len(set(zip(c.src.tolist(), c.dst.tolist()))) for c in cfgs], np.int64)
    return n, e


def algorithmic_bwd(w, K):
    """Algorithmic on-chip bytes of one adjoint call (cf_similarity_backward)
    over the workload's pairs, by the same rule as the forward: every operand
    a step needs read once, every result written once, 4 bytes each.

    Per pair (n_a n_b entries, e_a e_b successor pairs and as many
    predecessor pairs), with S = ceil(sqrt K) and R = (S - 1) * (number of
    segments but the last) recomputed steps:
      forward step (the first pass and each recomputed one):
        4 (2 e_a e_b + 2 n_a n_b)  -- gathered entries, (1-alpha) Ehat, Y written
      adjoint step (K of them):
        4 (2 e_a e_b + 2 n_a n_b)  -- Zbar gathered, Xbar written, Y_k read for <Xbar, X_k>
      + 4 (4 n_a n_b)              -- Ybar pass: Xbar, Y_{k+1} read; Zbar, Y_k written
      + 4 (4 e_a e_b)              -- edge terms: Zbar and Y_k at both ends of each pair of edges
    Returns (bytes, flops) with flops = 2 per gathered pair and edge term."""
    na, ea = _sizes(w.cfgs_a)
    nb, eb = _sizes(w.cfgs_b)
    a, b = w.pairs[:, 0], w.pairs[:, 1]
    nn = na[a] * nb[b]
    ee = ea[a] * eb[b]
    S = 1
    while S * S < K:
        S += 1
    nseg = (K - 1) // S + 1 if K > 0 else 0
    R = (S - 1) * max(nseg - 1, 0)
    fwd_step = 4 * (2 * ee + 2 * nn)
    adj_step = 4 * (2 * ee + 2 * nn) + 4 * 4 * nn + 4 * 4 * ee
    onchip = int(((K + R) * fwd_step + K * adj_step).sum())
    flops = int(((K + R) * (4 * ee + 5 * nn) + K * (4 * ee + 3 * nn + 6 * ee)).sum())
    return onchip, flops


def fwd_bwd_measure(dev, tune_cache, steps=5, warmup=3, bwd_tune=0):
    """The gradient workload: forward (scores + matchings) then the adjoint,
    each timed with CUDA events on the launching stream, L2 flushed before
    every step."""
    import torch

    from paper_1707_02423_gb300 import api

    w = workload("cfg4")
    fwd, bwd, P, tune = make_fwd_bwd(w, dev, tune_cache, bwd_tune)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        flush.zero_()
        fwd()
        bwd()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        fwd()
        e[1].record(stream)
        bwd()
        e[2].record(stream)
    torch.cuda.synchronize()
    step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in ev]))
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    bwd_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    onchip, flops = algorithmic_bwd(w, K_ITERS)
    return {"P": P, "step_ms": step_ms, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "bwd_bytes": onchip,
            "bwd_flops": flops, "tune": api.tune_info(tune)}


# A kernel configuration given on the command line (--tune) instead of the
# autotuner's pick, so that a profile can be taken of a named configuration.
FIXED_TUNE = 0


def pick_tune(pa, pb, pairs_np, omega, tune_cache):
    from paper_1707_02423_gb300 import api

    if FIXED_TUNE:
        return FIXED_TUNE
    return api.autotune(pa, pb, pairs_np, omega, ALPHA, K_ITERS, cache_path=tune_cache)[0]


def make_fwd_bwd(w, dev, tune_cache=None, bwd_tune=0):
    """(forward, adjoint, P, tune) callables of the gradient workload through
    the Python API, every buffer allocated up front."""
    import torch

    from paper_1707_02423_gb300 import _binding as B
    from paper_1707_02423_gb300 import api

    pairs_np = np.ascontiguousarray(w.pairs, np.int32)
    P = len(pairs_np)
    pa = api.Pack(w.cfgs_a, w.F, device=dev)
    pb = pa if w.shared else api.Pack(w.cfgs_b, w.F, device=dev)
    omega = torch.ones(w.F, dtype=torch.float32, device=dev)
    d_pairs = torch.from_numpy(pairs_np).to(dev)
    ws, bws = api.Workspace(dev), api.Workspace(dev)
    prm = B.params(ALPHA, K_ITERS)
    x_off, m_off = api.out_offsets(pa, pb, pairs_np)
    out = {"scores": torch.empty(P, dtype=torch.float32, device=dev),
           "match": torch.empty(int(m_off[-1]), dtype=torch.int32, device=dev)}
    tune = pick_tune(pa, pb, pairs_np, omega, tune_cache)
    ws_bytes = api.ws_size(pa, pb, pairs_np, B.params(ALPHA, K_ITERS, tune=tune))
    g = torch.ones(P, dtype=torch.float32, device=dev)
    grads = {"grad_w_a": torch.zeros(int(pa.info.n_user_edges), dtype=torch.float32, device=dev),
             "grad_omega": torch.zeros(w.F, dtype=torch.float32, device=dev)}
    if not w.shared:
        grads["grad_w_b"] = torch.zeros(int(pb.info.n_user_edges), dtype=torch.float32, device=dev)

    def fwd():
        api.similarity(pa, pb, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                       out=out, check_status=False, ws_bytes=ws_bytes, tune=tune)

    def bwd():
        for t in grads.values():  # the caller's accumulators start at zero every step
            t.zero_()
        api.similarity_backward(pa, pb, pairs_np, omega, out["match"], g, ALPHA, K_ITERS, ws=bws, out=grads,
                                d_pairs=d_pairs, check_status=False, tune=bwd_tune)
    return fwd, bwd, P, tune


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# The sources the forward kernels are built from; a committed profile counts
# only while their hash is the one it was taken with.
KERNEL_SOURCES = ("forward.cu", "iterate.cuh", "layout.h", "device_common.cuh")


def kernel_sources_sha256(csrc: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def profiled_traffic(csrc: str):
    """DRAM bytes per launch of the forward kernel from the committed ncu
    summary, if it was taken with the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "fwd_batched_kernel_cfg2.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", txt)
    h = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", txt)
    if m and h and h.group(1) == kernel_sources_sha256(csrc):
        return int(m.group(1))
    return None


def host_cores() -> int:
    """Host cores this process may run on (the oracle's process count), at most 32."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(32, n))


def _oracle_task(task):
    """One chunk of oracle work in a spawned worker: (kind, items) -> count.

    kind "score": steps 1-5 of a pair (X_K, greedy matching, score);
    "grad": the same and the reverse-mode gradient; "optimal": X_K and the
    maximum-weight assignment; "dist": the five resized Table 1 distances;
    "ward": a score matrix of seeded scores and its Ward linkage."""
    import oracle
    from oracle import distances as odist
    from oracle import ward as oward

    kind, items = task
    for it in items:
        if kind == "score":
            a, b, F = it
            oracle.pair_score(a, b, np.ones(F), ALPHA, K_ITERS)
        elif kind == "grad":
            a, b, F = it
            oracle.score_gradient(a, b, np.ones(F), ALPHA, K_ITERS, gbar=1.0)
        elif kind == "optimal":
            a, b, F = it
            oracle.optimal_match(oracle.similarity(a, b, np.ones(F), ALPHA, K_ITERS)["X"])
        elif kind == "dist":
            a, b, _ = it
            odist.pair_distances(a, b, 3.0)
        else:
            n_cfg, pairs, seed = it
            scores = np.random.default_rng(seed).uniform(1.0, 1.3, len(pairs))
            oward.linkage(oward.score_matrix(n_cfg, pairs, scores))
    return len(items)


class OraclePool:
    """The FP64 oracle as it stands on `cores` worker processes, one thread
    each, over independent units of work (the per-unit arithmetic is
    unchanged).  Each task carries its own CFGs, so no worker regenerates a
    workload.  The workers are spawned, not forked, so a pool started after
    CUDA initialisation is safe."""

    def __init__(self, cores: int):
        import multiprocessing as mp

        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)

    def run(self, kind, items, chunk: int = 1) -> int:
        parts = [(kind, items[i:i + chunk]) for i in range(0, len(items), chunk)]
        return sum(self.pool.map(_oracle_task, parts, chunksize=1))

    def close(self):
        self.pool.close()
        self.pool.join()


# the oracle's unit of work per workload (bench.py --workload ...)
ORACLE_KIND = {"cfg2": "score", "cfg3": "score", "cfg4": "grad", "cfg5": "score", "dist": "dist",
               "optimal": "optimal", "ward": "ward"}


def _oracle_items(name, w, idx):
    if ORACLE_KIND[name] == "ward":
        pairs = np.ascontiguousarray(w.pairs, np.int32)
        return [(len(w.cfgs_a), pairs, int(s)) for s in idx]
    return [(w.cfgs_a[int(w.pairs[p][0])], w.cfgs_b[int(w.pairs[p][1])], w.F) for p in idx]


def cpu_oracle(w, seconds: float, seed: int = 0, name: str = "cfg2"):
    """The oracle on all host cores, on a seeded random sample of the
    workload's units (pairs; for Ward, linkages of seeded scores) sized for
    about `seconds` of work (at most every pair): (rate, units timed,
    seconds, cores, what the sample is)."""
    cores = host_cores()
    kind = ORACLE_KIND[name]
    n_units = len(w.pairs) if kind != "ward" else 1 << 30
    order = (np.random.default_rng(seed).permutation(len(w.pairs)) if kind != "ward"
             else np.arange(4 * cores + 100000))
    pool = OraclePool(cores)
    try:
        pool.run(kind, _oracle_items(name, w, order[:cores]))  # starts every worker (spawn + imports), untimed
        t0 = time.perf_counter()
        pool.run(kind, _oracle_items(name, w, order[cores:3 * cores]))
        est = 2 * cores / (time.perf_counter() - t0)
        n = int(min(n_units - 3 * cores, max(2 * cores, est * seconds), len(order) - 3 * cores))
        # a workload smaller than the warm-up and the estimate is timed whole
        sample = order[3 * cores:3 * cores + n] if n >= cores else order[:min(len(order), n_units)]
        t0 = time.perf_counter()
        done = pool.run(kind, _oracle_items(name, w, sample))
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    what = {"score": "seeded random pairs of the workload (X_K, greedy matching, score)",
            "grad": "seeded random pairs of the workload (forward and reverse-mode gradient)",
            "optimal": "seeded random pairs of the workload (X_K and the maximum-weight assignment)",
            "dist": "seeded random pairs of the workload (resized transition matrices, five distances)",
            "ward": "score matrices of seeded scores of the workload's pairs and their Ward linkages"}[kind]
    desc = (f"{done} {what} in {dt:.1f} s, FP64 oracle (numpy/scipy) on {cores} processes of one thread each")
    return done / dt, done, dt, cores, desc


def dist_setup(n_gpus):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's figure (the job's time) when several ranks run."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(pairs_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job pairs/s: every rank runs its own replica of the workload
    (pairs are independent; no data-path collective), so the job completes
    world x pairs in the slowest rank's step time."""
    return world * pairs_per_rank / (ms_per_step * 1e-3)


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on all host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    cores = host_cores()
    order = np.random.default_rng(1).permutation(len(w.pairs))
    pool = OraclePool(cores)
    try:
        pool.run("score", _oracle_items("cfg2", w, order[:cores]))  # starts every worker, untimed
        t0 = time.perf_counter()
        pool.run("score", _oracle_items("cfg2", w, order[cores:3 * cores]))
        est = 2 * cores / (time.perf_counter() - t0)
        # size each step so that warmup + steps take about args.ref_seconds
        per_step = int(min(len(order), max(2 * cores, args.ref_seconds * est / (args.steps + args.warmup))))
        sample = order[:per_step]
        items = _oracle_items("cfg2", w, sample)
        for _ in range(args.warmup):
            pool.run("score", items)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.run("score", items)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    v = len(sample) * args.steps / dt
    desc = (f"{per_step} seeded random pairs of the workload per step, FP64 oracle (numpy/scipy) on {cores} "
            "processes of one thread each")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (oracle/isorank.py), host cores"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def timed_steps(step, steps, warmup, flush, stream):
    """Per-step CUDA-event times (ms) of `step`, L2 flushed before each step
    outside the events."""
    import torch

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def make_step(name, dev, tune_cache=None, bwd_tune=0):
    """The step of one workload through the Python API (kernel configuration
    from the autotuner): returns (step, n_pairs, launches_per_step, tune)."""
    import ctypes as C

    import torch

    from paper_1707_02423_gb300 import _binding as B
    from paper_1707_02423_gb300 import api

    w = workload(name)
    pairs_np = np.ascontiguousarray(w.pairs, np.int32)
    P = len(pairs_np)
    pa = api.Pack(w.cfgs_a, w.F, device=dev)
    pb = pa if w.shared else api.Pack(w.cfgs_b, w.F, device=dev)
    omega = torch.ones(w.F, dtype=torch.float32, device=dev)
    d_pairs = torch.from_numpy(pairs_np).to(dev)
    ws = api.Workspace(dev)
    prm = B.params(ALPHA, K_ITERS)
    x_off, m_off = api.out_offsets(pa, pb, pairs_np)
    out = {"scores": torch.empty(P, dtype=torch.float32, device=dev),
           "match": torch.empty(int(m_off[-1]), dtype=torch.int32, device=dev)}
    tune = pick_tune(pa, pb, pairs_np, omega, tune_cache)
    # kernels per forward call: the three plan kernels, the persistent forward
    # and, under a cluster tune, the cluster-tier kernel; per adjoint call: the
    # three plan kernels, the accumulator reset, the adjoint and the scatter
    n_fwd = 4 + (1 if api.tune_info(tune)["cluster"] >= 2 else 0) + \
        (1 if api.tune_info(tune)["matching"].startswith("ranked, sequential") else 0)
    n_bwd = 3 + 1 + 2 + (1 if w.shared else 2)  # plan, zero, large-pair and resident kernels, scatter
    if name == "dist":  # the C ABI directly, every buffer allocated before the timed region
        L = B.lib()
        n = C.c_size_t(0)
        B.check(L.cf_distances_ws_size(P, C.byref(n)))
        dws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
        dout = torch.empty(P, 5, dtype=torch.float32, device=dev)
        st = int(torch.cuda.current_stream().cuda_stream)

        def step():
            B.check(L.cf_distances(pa.dev.data_ptr(), pb.dev.data_ptr(), d_pairs.data_ptr(), P, 3.0,
                                   B.CF_DIST_SCALE01, dout.data_ptr(), dws.data_ptr(), dws.numel(), st))
        return step, P, 3, tune
    if name == "optimal":
        ws_bytes = api.ws_size(pa, pb, pairs_np, B.params(ALPHA, K_ITERS, match_mode=B.CF_MATCH_OPTIMAL))
        out["X"] = torch.empty(int(x_off[-1]), dtype=torch.float32, device=dev)

        def step():
            api.similarity(pa, pb, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                           out=out, check_status=False, ws_bytes=ws_bytes, tune=tune, optimal=True)
        return step, P, n_fwd + 1, tune
    if name == "ward":  # the pair scores are computed once, outside the step
        api.similarity(pa, pb, pairs_np, omega, ALPHA, K_ITERS, ws=ws, d_pairs=d_pairs, out=out, tune=tune)
        L = B.lib()
        n_cfg = len(w.cfgs_a)
        S = torch.empty(n_cfg, n_cfg, dtype=torch.float32, device=dev)
        sstat = torch.empty(1, dtype=torch.int32, device=dev)
        nb = C.c_size_t(0)
        B.check(L.cf_ward_ws_size(n_cfg, C.byref(nb)))
        wws = torch.empty(int(nb.value), dtype=torch.uint8, device=dev)
        merge = torch.empty(n_cfg - 1, 2, dtype=torch.int32, device=dev)
        height = torch.empty(n_cfg - 1, dtype=torch.float32, device=dev)
        size = torch.empty(n_cfg - 1, dtype=torch.int32, device=dev)
        st = int(torch.cuda.current_stream().cuda_stream)

        def step():
            B.check(L.cf_score_matrix(d_pairs.data_ptr(), out["scores"].data_ptr(), P, n_cfg, n_cfg, 1, S.data_ptr(),
                                      sstat.data_ptr(), st))
            B.check(L.cf_ward(S.data_ptr(), n_cfg, n_cfg, merge.data_ptr(), height.data_ptr(), size.data_ptr(),
                              wws.data_ptr(), wws.numel(), st))
        return step, 1, 4, tune
    if name in ("cfg2", "cfg3"):
        ws_bytes = api.ws_size(pa, pb, pairs_np, B.params(ALPHA, K_ITERS, tune=tune))

        def step():
            api.similarity(pa, pb, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                           out=out, check_status=False, ws_bytes=ws_bytes, tune=tune)
        return step, P, n_fwd, tune
    if name == "cfg4":
        fwd, bwd, _, tune = make_fwd_bwd(w, dev, tune_cache, bwd_tune)

        def step():
            fwd()
            bwd()
        return step, P, n_fwd + n_bwd + (2 if w.shared else 3), tune
    # cfg5: scores of every query-corpus pair, top-16 per query, matchings of
    # the winners -- one CUDA graph: the winners' pair list is built on the
    # device from the top-k indices (cf_topk_pairs), so nothing returns to the
    # host between the steps
    step, P, launches = make_query_step(w, pa, pb, omega, d_pairs, ws, tune)
    return step, P, launches, tune


def make_query_step(w, pa, pb, omega, d_pairs, ws, tune):
    """The query step (scores of all query x corpus pairs, top-k per query, the
    winners' matchings) captured once as one CUDA graph; returns
    (replay, pairs, kernels per step) -- the replay also exposes the buffers as
    attributes (scores, top, idx, win, win_scores, win_match)."""
    import torch

    from paper_1707_02423_gb300 import _binding as B
    from paper_1707_02423_gb300 import api

    dev = pa.dev.device
    nq, nc, k = w.meta["n_query"], w.meta["n_corpus"], w.meta["top_k"]
    pairs_np = np.ascontiguousarray(w.pairs, np.int32)
    P = len(pairs_np)
    prm = B.params(ALPHA, K_ITERS, tune=tune)
    ws_bytes = api.ws_size(pa, pb, pairs_np, prm)
    scores = torch.empty(P, dtype=torch.float32, device=dev)
    top = torch.empty(nq, k, dtype=torch.float32, device=dev)
    idx = torch.empty(nq, k, dtype=torch.int32, device=dev)
    win = torch.empty(nq * k, 2, dtype=torch.int32, device=dev)
    mws = api.Workspace(dev)
    mws_bytes = api.ws_size_any(pa, pb, nq * k, prm)
    win_scores = torch.empty(nq * k, dtype=torch.float32, device=dev)
    win_match = torch.empty(int(k * pa.n_blocks[:nq].sum()), dtype=torch.int32, device=dev)

    def body():
        api.similarity(pa, pb, pairs_np, omega, ALPHA, K_ITERS, want_match=False, ws=ws, d_pairs=d_pairs,
                       out={"scores": scores}, check_status=False, ws_bytes=ws_bytes, tune=tune)
        api.topk(scores.view(nq, nc), k, out=(top, idx))
        api.topk_pairs(idx, out=win)
        api.similarity_dev(pa, pb, win, omega, ALPHA, K_ITERS, scores=win_scores, match=win_match, ws=mws,
                           ws_bytes=mws_bytes, tune=tune)

    body()  # every kind of call once uncaptured (first use sets kernel attributes)
    torch.cuda.synchronize()
    g = api.Graph(dev)
    with g.capture():
        body()
    n_fwd = 4 + (1 if api.tune_info(tune)["cluster"] >= 2 else 0) + \
        (1 if api.tune_info(tune)["matching"].startswith("ranked, sequential") else 0)

    def replay():
        g.launch()
    replay.graph, replay.scores, replay.top, replay.idx = g, scores, top, idx
    replay.win, replay.win_scores, replay.win_match = win, win_scores, win_match
    return replay, P, 2 * n_fwd + 2


def onchip_peak(kind, f_mhz=None):
    """A measured on-chip peak (cf_probe) in GB/s at the SM clock f_mhz (the
    probe's own clock when None), with its description."""
    import torch

    from paper_1707_02423_gb300 import _binding as B
    from paper_1707_02423_gb300 import api

    pr = api.probe(kind, reps=3)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    f = f_mhz or pr["sm_mhz"]
    name = {B.CF_PROBE_SMEM: "shared-memory loads", B.CF_PROBE_L2: "L2 re-reads (volatile, L1 bypassed)",
            B.CF_PROBE_DSMEM: "distributed-shared-memory loads (2-CTA clusters)"}.get(kind, "FP32 FMA")
    unit = "B" if kind != B.CF_PROBE_FP32 else "FLOP"
    peak = pr["per_clk_sm"] * n_sm * f * 1e6 / 1e9
    desc = (f"of measured: cf_probe {name} {pr['per_clk_sm']:.1f} {unit}/clk/SM ({pr['rate'] / 1e9:.0f} G{unit}/s "
            f"at {pr['sm_mhz']:.0f} MHz) x {n_sm} SMs x {f:.0f} MHz")
    return peak, desc, pr


def prune_demo(w, scores):
    """Query pruning (the next row of the query workload), measured: a
    corpus CFG could be skipped for query q only if an upper bound on s(q, c)
    fell below q's k-th best score.  The only admissible bound the measure
    gives is s <= sqrt(min(n_q, n_c)) (a sum of min(n_q, n_c) entries of a
    nonnegative X with |X|_F = 1, Cauchy-Schwarz; tight for a general X);
    an attribute-only term cannot do better, because the attribute term's
    share of X is at most 1 - alpha and the propagation term is unbounded by
    it.  Returns the counts of this run."""
    nq, nc, k = w.meta["n_query"], w.meta["n_corpus"], w.meta["top_k"]
    S = np.asarray(scores, np.float64).reshape(nq, nc)
    kth = -np.sort(-S, axis=1)[:, k - 1]
    n_q = np.array([c.n for c in w.cfgs_a], np.float64)
    n_c = np.array([c.n for c in w.cfgs_b], np.float64)
    bound = np.sqrt(np.minimum(n_q[:, None], n_c[None, :]))
    return {"bound": "s <= sqrt(min(n_q, n_c))", "pairs": int(S.size),
            "prunable_pairs": int((bound < kth[:, None]).sum()),
            "smallest_bound": float(bound.min()), "largest_kth_best_score": float(kth.max()),
            "largest_score": float(S.max())}


def run_workload(args):
    """--workload cfg3 / cfg4 / cfg5 / dist / optimal / ward: one JSON line for
    that workload alone, with the oracle timed on all host cores beside it,
    and the roofline of the bandwidth-bound ones."""
    import torch

    from paper_1707_02423_gb300 import _binding as B
    from paper_1707_02423_gb300 import api

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    step, P, launches, tune = make_step(args.workload, dev, args.tune_cache)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with ClockSampler(local) as clk:
        ms = timed_steps(step, args.steps, args.warmup, flush, stream)
    tot = max_over_ranks(float(sum(ms)), world, dev)
    if rank != 0:
        return
    mps = tot / args.steps
    unit = UNITS.get(args.workload, UNIT)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": job_rate(P, world, mps), "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "pairs": P,
                   "l2": "flushed between steps (256 MiB write, outside the step events)",
                   "tune": api.tune_info(tune)},
        "gpu_launches": launches * args.steps, "clocks": clocks,
    }
    w = workload(args.workload)
    if args.workload in ("cfg3", "cfg4", "cfg5"):
        # algorithmic on-chip bytes of the step (the forward's rule; the
        # adjoint's for cfg4) over the step time, against the measured peak of
        # the memory the iterations run from: L2 for the large CFGs (X in
        # scratch slots), shared memory for the others
        onchip = algorithmic(w, K_ITERS)[0]
        if args.workload == "cfg4":
            onchip += algorithmic_bwd(w, K_ITERS)[0]
        kind = B.CF_PROBE_L2 if args.workload == "cfg3" else B.CF_PROBE_SMEM
        peak, desc, _ = onchip_peak(kind, clocks["sm_mhz"])
        achieved = onchip / (mps * 1e-3) / 1e9
        line["roofline"] = {"bound": "l2" if kind == B.CF_PROBE_L2 else "smem",
                            "kernel": {"cfg3": "fwd_batched_kernel / fwd_cluster_kernel (global-memory tier)",
                                       "cfg4": "the whole forward + adjoint step",
                                       "cfg5": "the whole query step (forward kernels, top-k, winners' matching)"}[
                                           args.workload],
                            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                            "traffic": None, "algorithmic_bytes_per_step": onchip, "peak_source": desc}
    if args.workload == "cfg5":
        line["pruning"] = prune_demo(w, step.scores.cpu().numpy())
    v, n, dt, cores, desc = cpu_oracle(w, args.cpu_seconds, name=args.workload)
    line["cpu_baseline"] = {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": desc}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import ctypes as C

    import torch

    from paper_1707_02423_gb300 import _binding as B
    from paper_1707_02423_gb300 import api

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = workload()
    P = len(w.pairs)
    pairs_np = np.ascontiguousarray(w.pairs, np.int32)
    gather = None
    if world > 1:
        # the job: one copy of the workload's pair list per rank, partitioned
        # across the ranks by LPT cost (each rank gets about P pairs, so the
        # per-GPU work stays fixed as N grows), the pack replicated, and the
        # scores all-gathered back into job order at the end of every step
        from paper_1707_02423_gb300 import shard

        job = np.tile(pairs_np, (world, 1))
        ns = np.array([c.n for c in w.cfgs_a], np.int64)
        es = np.array([len(set(zip(c.src.tolist(), c.dst.tolist()))) for c in w.cfgs_a], np.int64)
        parts = shard.lpt_partition(shard.pair_costs(ns, ns, es, es, job), world)
        pairs_np = np.ascontiguousarray(job[parts[rank]], np.int32)
        gather = shard.ScoreGather(parts, len(job), dev)
        P = len(pairs_np)
    pack = api.Pack(w.cfgs_a, w.F, device=dev)
    omega = torch.ones(w.F, dtype=torch.float32, device=dev)
    d_pairs = torch.from_numpy(pairs_np).to(dev)
    ws = api.Workspace(dev)
    prm = B.params(ALPHA, K_ITERS)
    x_off, m_off = api.out_offsets(pack, pack, pairs_np)
    out = {"scores": torch.empty(P, dtype=torch.float32, device=dev),
           "match": torch.empty(int(m_off[-1]), dtype=torch.int32, device=dev)}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # on-chip peak the iteration kernel is bound by, measured on this GPU
    smem_probe = api.probe(B.CF_PROBE_SMEM, reps=3)
    # kernel configuration: the autotuner's pick for this workload (cached per device and workload)
    tune_ms = None
    if FIXED_TUNE:
        tune = FIXED_TUNE
    else:
        tune, tune_ms = api.autotune(pack, pack, pairs_np, omega, ALPHA, K_ITERS, cache_path=args.tune_cache)
    prm.tune = tune
    ws_bytes = api.ws_size(pack, pack, pairs_np, prm)  # with room for deferred matching steps under such a tune
    deferred = api.tune_info(tune)["matching"].startswith("ranked, sequential")

    def sim(flags):
        api.similarity(pack, pack, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                       out=out, check_status=False, flags=flags, ws_bytes=ws_bytes, tune=tune)

    # one step = the plan graph (workspace reset + 3 plan kernels) and the
    # forward graph (queue reset + the persistent kernel), each captured once
    sim(B.CF_FLAG_PLAN_ONLY)
    sim(B.CF_FLAG_REUSE_PLAN)
    torch.cuda.synchronize()
    g_plan, g_fwd = api.Graph(dev), api.Graph(dev)
    with g_plan.capture():
        sim(B.CF_FLAG_PLAN_ONLY)
    with g_fwd.capture():
        sim(B.CF_FLAG_REUSE_PLAN)

    for _ in range(args.warmup):
        flush.zero_()
        g_plan.launch(stream)
        g_fwd.launch(stream)
    B.check(B.lib().cf_status_check(ws.get(ws_bytes).data_ptr(), int(stream.cuda_stream)))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()  # outside the step's events
            ev[i][0].record(stream)
            g_plan.launch(stream)
            ev[i][1].record(stream)
            g_fwd.launch(stream)
            if gather is not None:
                gather(out["scores"])  # the exchange step: every rank gets the job's scores
            ev[i][2].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    fwd_ms = [e[1].elapsed_time(e[2]) for e in ev]
    tot_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    B.check(B.lib().cf_status_check(ws.get(ws_bytes).data_ptr(), int(stream.cuda_stream)))
    ms_per_step = tot_ms / args.steps
    value = job_rate(len(w.pairs), world, ms_per_step)  # world copies of the workload per step

    # ---- per-pair form: one launch per pair, same math
    pp_steps = 2
    for _ in range(1):
        api.similarity(pack, pack, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                       out=out, check_status=False, per_pair=True, ws_bytes=ws_bytes, tune=tune)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(pp_steps):
        flush.zero_()
        api.similarity(pack, pack, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                       out=out, check_status=False, per_pair=True, ws_bytes=ws_bytes, tune=tune)
    e1.record(stream)
    torch.cuda.synchronize()
    pp_ms = e0.elapsed_time(e1) / pp_steps
    # the same launches spread over 32 streams: what remains of the gap is
    # per-launch cost and one pair per SM, not the serialisation
    api.similarity(pack, pack, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs, out=out,
                   check_status=False, per_pair=True, flags=B.CF_FLAG_PER_PAIR_STREAMS, tune=tune)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(pp_steps):
        flush.zero_()
        api.similarity(pack, pack, pairs_np, omega, ALPHA, K_ITERS, want_match=True, ws=ws, d_pairs=d_pairs,
                       out=out, check_status=False, per_pair=True, flags=B.CF_FLAG_PER_PAIR_STREAMS, tune=tune)
    e1.record(stream)
    torch.cuda.synchronize()
    pps_ms = e0.elapsed_time(e1) / pp_steps

    # ---- forward + adjoint on the gradient workload (256 pairs, n 10-300)
    fb = fwd_bwd_measure(dev, args.tune_cache)
    fb_mps = fb["step_ms"]
    fb_p = fb["P"]

    # ---- end to end through the C ABI with host buffers: build + upload the
    # pack from the host CFG arrays, upload the pairs from pinned memory,
    # compute, read scores and matchings back into pinned memory
    L = B.lib()
    pairs_pin = torch.from_numpy(pairs_np).pin_memory()
    sc_pin = torch.empty(P, dtype=torch.float32).pin_memory()
    mt_pin = torch.empty(int(m_off[-1]), dtype=torch.int32).pin_memory()
    dpack = torch.empty(pack.host.size, dtype=torch.uint8, device=dev)
    wbuf = ws.get(ws_bytes)
    e2e_steps = max(3, min(20, args.steps // 10))
    e2e_ts = []
    for it in range(e2e_steps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.check(L.cf_pack_cfgs(pack._views, pack.n_cfgs, w.F, dpack.data_ptr(), dpack.numel(),
                               int(stream.cuda_stream)))
        d_pairs.copy_(pairs_pin, non_blocking=True)
        B.check(L.cf_similarity(dpack.data_ptr(), dpack.data_ptr(), d_pairs.data_ptr(), P, C.byref(prm),
                                omega.data_ptr(), None, out["scores"].data_ptr(), out["match"].data_ptr(),
                                wbuf.data_ptr(), ws_bytes, int(stream.cuda_stream)))
        sc_pin.copy_(out["scores"], non_blocking=True)
        mt_pin.copy_(out["match"], non_blocking=True)
        torch.cuda.synchronize()
        if it >= 2:
            e2e_ts.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_ts)
    h2d = int(pack.host.size + pairs_np.nbytes)
    d2h = int(sc_pin.numel() * 4 + mt_pin.numel() * 4)

    if rank != 0:
        return
    import dataclasses

    # this rank's pairs (the whole workload at N = 1)
    onchip, flops, x_elems, m_elems = algorithmic(dataclasses.replace(w, pairs=pairs_np), K_ITERS)
    fwd_mean_s = statistics.mean(fwd_ms) * 1e-3
    clk = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    f_mhz = clk["sm_mhz"] or smem_probe["sm_mhz"]
    # measured shared-memory bytes per clock per SM, at the SM clock sampled during the timed region
    smem_peak_gbs = smem_probe["per_clk_sm"] * n_sm * f_mhz * 1e6 / 1e9
    achieved = onchip / fwd_mean_s / 1e9
    peaks = measured_peaks()
    hbm_bytes = int(pack.host.size + pairs_np.nbytes + P * 4 + m_elems * 4)
    traffic = profiled_traffic(os.path.join(ROOT, "paper_1707_02423_gb300", "csrc"))
    cpu_baseline = None  # the oracle is timed at N = 1 only
    if world == 1:
        cpu_v, cpu_n, cpu_dt, cpu_cores, cpu_desc = cpu_oracle(w, args.cpu_seconds)
        cpu_baseline = {"value": cpu_v, "unit": UNIT, "cores": cpu_cores, "kind": "oracle", "sample": cpu_desc}
    probes = {}
    for nm, kind in (("l2", B.CF_PROBE_L2), ("dsmem", B.CF_PROBE_DSMEM), ("fp32", B.CF_PROBE_FP32)):
        pr = api.probe(kind, reps=3)
        probes[nm] = {"per_clk_sm": pr["per_clk_sm"], "rate": pr["rate"], "sm_mhz": pr["sm_mhz"],
                      "unit": "FLOP/s" if nm == "fp32" else "B/s"}
    probes["smem"] = {"per_clk_sm": smem_probe["per_clk_sm"], "rate": smem_probe["rate"],
                      "sm_mhz": smem_probe["sm_mhz"], "unit": "B/s"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs": len(w.pairs) * world, "pairs_per_rank": P,
                   "parallelism": (f"dp{world}: one copy of the pair list per rank, partitioned over the ranks by "
                                   "LPT cost, pack replicated, scores all-gathered every step") if world > 1 else
                                  "one GPU", "n_cfgs": len(w.cfgs_a), "F": w.F, "K": K_ITERS,
                   "alpha": ALPHA, "l2": "flushed between steps (256 MiB write, outside the step events)",
                   "step": "two CUDA-graph launches: plan (workspace reset + 3 kernels), forward (queue reset + "
                           "persistent kernel); sum of per-step CUDA events",
                   "tune": {**api.tune_info(tune), "autotune_sample_ms": tune_ms}},
        "roofline": {"bound": "smem",
                     "kernel": "fwd_batched_kernel + match_deferred_kernel (the forward graph)" if deferred
                     else "fwd_batched_kernel", "achieved": achieved,
                     "peak": smem_peak_gbs, "unit": "GB/s", "frac": achieved / smem_peak_gbs,
                     "traffic": traffic,
                     "peak_source": f"of measured: cf_probe shared-memory loads {smem_probe['per_clk_sm']:.1f} "
                                    f"B/clk/SM ({smem_probe['rate'] / 1e9:.0f} GB/s at {smem_probe['sm_mhz']:.0f} MHz) "
                                    f"x {n_sm} SMs x {f_mhz:.0f} MHz (median SM clock sampled in the timed region)",
                     "algorithmic_bytes_per_launch": onchip, "kernel_ms": fwd_mean_s * 1e3,
                     "flops_per_launch": flops, "achieved_tflops_fp32": flops / fwd_mean_s / 1e12,
                     "hbm": {"algorithmic_bytes_per_step": hbm_bytes,
                             "achieved_gbs": hbm_bytes / (ms_per_step * 1e-3) / 1e9,
                             "peak_gbs": peaks.get("hbm_gbs"),
                             "frac": (hbm_bytes / (ms_per_step * 1e-3) / 1e9) / peaks["hbm_gbs"]
                             if peaks.get("hbm_gbs") else None, "peak_source": "MEASURED_PEAKS.json (of measured)"}},
        "fwd_bwd": {"value": fb_p / (fb_mps * 1e-3), "unit": UNIT, "ms_per_step": fb_mps,
                    "workload": WORKLOADS["cfg4"], "fwd_ms": fb["fwd_ms"], "bwd_ms": fb["bwd_ms"],
                    "roofline": {"bound": "smem", "kernel": "bwd_big_kernel + bwd_res_kernel (concurrent, the "
                                 "whole adjoint call)",
                                 "achieved": fb["bwd_bytes"] / (fb["bwd_ms"] * 1e-3) / 1e9,
                                 "peak": smem_peak_gbs, "unit": "GB/s",
                                 "frac": fb["bwd_bytes"] / (fb["bwd_ms"] * 1e-3) / 1e9 / smem_peak_gbs,
                                 "traffic": None, "algorithmic_bytes_per_launch": fb["bwd_bytes"],
                                 "flops_per_launch": fb["bwd_flops"], "kernel_ms": fb["bwd_ms"],
                                 "peak_source": "of measured: the same shared-memory peak as the forward's line"}},
        "per_pair": {"value": P / (pp_ms * 1e-3), "unit": UNIT, "ms_per_step": pp_ms, "launches_per_step": P,
                     "speedup_batched_over_per_pair": pp_ms / ms_per_step,
                     "over_32_streams": {"value": P / (pps_ms * 1e-3), "ms_per_step": pps_ms,
                                         "speedup_batched_over_it": pps_ms / ms_per_step}},
        "cpu_baseline": cpu_baseline,
        "e2e": {"value": world * P / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3,
                "what": "cf_pack_cfgs (host build + copy) + pinned pair upload + cf_similarity + pinned "
                        "readback of scores and matchings, wall clock"},
        # per step: the three plan kernels, the persistent forward, the
        # cluster-tier kernel when the tune has one, and the deferred
        # matching steps when the tune defers them
        "gpu_launches": (4 + (1 if api.tune_info(tune)["cluster"] >= 2 else 0) + (1 if deferred else 0)) * args.steps,
        "clocks": clk,
        "probes": probes,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="--impl reference: oracle work per run (warmup + steps), in seconds")
    ap.add_argument("--workload", default="cfg2", choices=sorted(WORKLOADS))
    ap.add_argument("--tune", type=int, default=0,
                    help="kernel configuration id for the forward (0: the autotuner's pick)")
    ap.add_argument("--tune-cache", default=os.environ.get("CF_AUTOTUNE_CACHE") or
                    os.path.join(tempfile.gettempdir(), "cfsim_autotune.cache"))
    ap.add_argument("--pairs", type=int, default=0,
                    help="--workload cfg3: only the first N pairs (a smaller case for profiling)")
    args = ap.parse_args()
    global FIXED_TUNE, PAIR_LIMIT
    FIXED_TUNE = args.tune
    PAIR_LIMIT = args.pairs if args.workload == "cfg3" else 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "cfg2":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
