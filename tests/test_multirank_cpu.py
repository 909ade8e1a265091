"""The N > 1 path on CPU ranks (gloo, world size 2): the timing reduction of
bench.py (the slowest rank's time), the reference arm printing on rank 0
only, and the partitioned form of paper_1707_02423_gb300.shard (LPT pair
partition, all-gathered scores, merged top-k, all-reduced gradients) with
every rank's compute stubbed by the FP64 oracle."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        rate = bench.job_rate(100, world, slow)
        q.put((rank, slow, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, slow, rate in got:
        assert slow == 15.0  # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 100 / 15e-3)  # 200 pairs in 15 ms


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(19900, 1, 10.0) == pytest.approx(1.99e6)


def test_reference_arm_on_a_nonzero_rank_prints_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_line_on_rank_zero():
    import json

    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--ref-seconds", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "pairs/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1



# ---------------------------------------------------------------------------
# The partitioned form (paper_1707_02423_gb300.shard) on gloo CPU ranks, with
# every rank's compute stubbed by the FP64 oracle: the LPT partition covers
# every pair exactly once, and the all-gathered scores, the merged top-k and
# the all-reduced gradients equal what one rank computes over all pairs.

def _distinct_edges(cfgs):
    import numpy as np

    return np.array([len(set(zip(c.src.tolist(), c.dst.tolist()))) for c in cfgs], np.int64)


def _select_lexsort(scores, ids, k):
    """Reference selection: k largest per row, ties to the smaller id."""
    import numpy as np

    s, i = scores.numpy(), ids.numpy()
    top = np.zeros((s.shape[0], k), s.dtype)
    out = np.zeros((s.shape[0], k), np.int64)
    for q in range(s.shape[0]):
        key = np.where(i[q] < 0, np.iinfo(np.int64).max, i[q])
        o = np.lexsort((key, -s[q]))[:k]
        top[q], out[q] = s[q][o], i[q][o]
    return torch.from_numpy(top), torch.from_numpy(out)


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    from gen import config1, config5
    from paper_1707_02423_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = config1()
        n = np.array([c.n for c in w.cfgs_a])
        e = _distinct_edges(w.cfgs_a)
        P = len(w.pairs)
        parts = shard.lpt_partition(shard.pair_costs(n, n, e, e, w.pairs), world)
        mine = parts[rank]
        om = np.linspace(0.5, 1.5, w.F)
        loc = torch.tensor([oracle.pair_score(w.cfgs_a[a], w.cfgs_a[b], om)[2] for a, b in w.pairs[mine]],
                           dtype=torch.float64)
        full = shard.ScoreGather(parts, P, "cpu", torch.float64)(loc)
        # gradients of every pair's score (upstream 1), summed over the ranks
        ua = np.concatenate([[0], np.cumsum([len(c.src) for c in w.cfgs_a])])
        gw = torch.zeros(int(ua[-1]), dtype=torch.float64)
        go = torch.zeros(w.F, dtype=torch.float64)
        for a, b in w.pairs[mine]:
            g = oracle.score_gradient(w.cfgs_a[a], w.cfgs_a[b], om)
            gw[ua[a]:ua[a + 1]] += torch.from_numpy(g["grad_w_a"])
            gw[ua[b]:ua[b + 1]] += torch.from_numpy(g["grad_w_b"])
            go += torch.from_numpy(g["grad_omega"])
        shard.allreduce_sum(gw, go)
        # query workload: every rank scores its part of the pairs, keeps each
        # query's local top-k among its corpus entries, and the candidates merge
        wq = config5(2, 24)
        k = 4
        nq_, nc_ = wq.meta["n_query"], wq.meta["n_corpus"]
        nqa = np.array([c.n for c in wq.cfgs_a])
        ncb = np.array([c.n for c in wq.cfgs_b])
        qparts = shard.lpt_partition(shard.pair_costs(nqa, ncb, _distinct_edges(wq.cfgs_a),
                                                      _distinct_edges(wq.cfgs_b), wq.pairs), world)
        S = np.full((nq_, nc_), -np.inf)
        for p in qparts[rank]:
            a, b = wq.pairs[p]
            S[a, b] = oracle.pair_score(wq.cfgs_a[a], wq.cfgs_b[b], np.ones(wq.F))[2]
        ltop, lidx = _select_lexsort(torch.from_numpy(S), torch.arange(nc_).repeat(nq_, 1), k)
        lidx[torch.isinf(ltop)] = -1
        top, ids = shard.merge_topk(ltop, lidx, k, select=_select_lexsort)
        q.put((rank, [p.tolist() for p in parts], full.numpy(), gw.numpy(), go.numpy(), top.numpy(), ids.numpy(),
               [p.tolist() for p in qparts]))
    finally:
        dist.destroy_process_group()


def test_partitioned_form_with_gloo():
    import numpy as np
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import oracle
    from gen import config1, config5

    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(qu.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0

    w = config1()
    P = len(w.pairs)
    om = np.linspace(0.5, 1.5, w.F)
    ref = np.array([oracle.pair_score(w.cfgs_a[a], w.cfgs_a[b], om)[2] for a, b in w.pairs])
    ua = np.concatenate([[0], np.cumsum([len(c.src) for c in w.cfgs_a])])
    gw = np.zeros(ua[-1])
    go = np.zeros(w.F)
    for a, b in w.pairs:
        g = oracle.score_gradient(w.cfgs_a[a], w.cfgs_a[b], om)
        gw[ua[a]:ua[a + 1]] += g["grad_w_a"]
        gw[ua[b]:ua[b + 1]] += g["grad_w_b"]
        go += g["grad_omega"]
    wq = config5(2, 24)
    S = np.array([oracle.pair_score(wq.cfgs_a[a], wq.cfgs_b[b], np.ones(wq.F))[2] for a, b in wq.pairs])
    S = S.reshape(wq.meta["n_query"], wq.meta["n_corpus"])

    parts = got[0][1]
    assert got[1][1] == parts  # both ranks derive the same partition
    allp = sorted(parts[0] + parts[1])
    assert allp == list(range(P))  # every pair exactly once
    assert min(len(parts[0]), len(parts[1])) > 0
    qp = got[0][7]
    assert sorted(qp[0] + qp[1]) == list(range(len(wq.pairs)))
    for rank, _, full, g_w, g_o, top, ids, _ in got:
        assert np.allclose(full, ref, rtol=0, atol=1e-12)  # gathered in pair order
        assert np.allclose(g_w, gw, rtol=1e-12, atol=1e-15)
        assert np.allclose(g_o, go, rtol=1e-12, atol=1e-15)
        for q in range(S.shape[0]):
            o = np.lexsort((np.arange(S.shape[1]), -S[q]))[:4]
            assert np.array_equal(ids[q], o)
            assert np.array_equal(top[q], S[q][o])


def test_lpt_partition_balance():
    import numpy as np

    sys.path.insert(0, ROOT)
    from paper_1707_02423_gb300 import shard

    rng = np.random.default_rng(0)
    costs = rng.integers(1, 10000, 997)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(len(costs)))
        loads = np.array([costs[p].sum() for p in parts])
        # LPT: the most loaded rank exceeds the least by at most one pair's cost
        assert loads.max() - loads.min() <= costs.max()
