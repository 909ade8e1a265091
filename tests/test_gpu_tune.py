"""Every kernel configuration (cf_params.tune) against the FP64 oracle, and
the autotuner (cf_autotune) with its cache file."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from _helpers import ATOL_S, TIE_EPS, greedy_margin, valid_matching  # noqa: E402
from gen import config2  # noqa: E402
from paper_1707_02423_gb300 import _binding as B  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def wl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()
    # 22 CFGs, n in [8, 120]: warp-, quarter-, CTA- and global-class pairs
    w = config2(22)
    om = np.linspace(0.6, 1.4, w.F)
    ref = []
    for a, b in w.pairs:
        X = oracle.similarity(w.cfgs_a[a], w.cfgs_a[b], om, 0.8, 40)["X"]
        m, s = oracle.greedy_match(X)
        ref.append((greedy_margin(X) > TIE_EPS, m, s, X))
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    return w, pa, torch.tensor(om, dtype=torch.float32, device=DEV), ref


NT = 240
DEFER = [181, 182, 183, 198, 228]  # matching steps deferred: 1024 / 512 / 768 threads; 768 with 2- and 8-CTA clusters


def test_tune_table():
    L = B.lib()
    assert L.cf_num_tunes() == NT
    seen = set()
    for t in range(0, NT + 1):
        d = api.tune_info(t)
        assert d["threads_per_cta"] in (512, 768, 1024)
        assert d["smallest_group"] in (32, *(d["threads_per_cta"] // k for k in (8, 4, 2, 1)))
        assert d["cluster"] in (0, 2, 4, 8)
        if t > 0:
            seen.add((d["threads_per_cta"], d["smallest_group"], d["matching"], d["cluster"]))
    assert len(seen) == NT
    assert api.tune_info(0) == {**api.tune_info(1), "tune": 0}


@pytest.mark.parametrize("tune", list(range(1, NT + 1, 7)) + [2, 3, 6, 9, 12, 15, 45, 46, 47, 90, 92, 135, 136, 180]
                         + DEFER)
def test_every_tune_matches_oracle(wl, tune):
    w, pa, om, ref = wl
    res = api.similarity(pa, pa, w.pairs, om, 0.8, 40, want_match=True, tune=tune)
    scores = res.scores.cpu().numpy()
    match = res.match.cpu().numpy()
    for p, (a, b) in enumerate(w.pairs):
        clear, m_ref, s_ref, X = ref[p]
        m = match[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, w.cfgs_a[a].n, w.cfgs_a[b].n), p
        if clear:
            assert np.array_equal(m, m_ref), (tune, p)
            assert abs(float(scores[p]) - s_ref) <= ATOL_S, (tune, p)
        else:
            s_own = sum(X[i, m[i]] for i in range(len(m)) if m[i] >= 0)
            assert abs(float(scores[p]) - s_own) <= ATOL_S, (tune, p)


def test_autotune_picks_a_tune_and_caches_it(wl, tmp_path):
    w, pa, om, ref = wl
    cache = str(tmp_path / "tune.cache")
    t1, ms1 = api.autotune(pa, pa, w.pairs, om, cache_path=cache)
    assert 1 <= t1 <= NT and ms1 > 0.0
    lines = open(cache).read().split("\n")
    assert len([x for x in lines if x.strip()]) == 1
    key, tid, ms = lines[0].split()
    assert int(tid) == t1 and "sm=" in key and "K=40" in key
    t2, ms2 = api.autotune(pa, pa, w.pairs, om, cache_path=cache)  # cache hit: no timing
    assert (t2, round(ms2, 4)) == (t1, round(ms1, 4))
    assert len([x for x in open(cache).read().split("\n") if x.strip()]) == 1
    # a different K is a different key
    t3, _ = api.autotune(pa, pa, w.pairs, om, K=20, cache_path=cache)
    assert 1 <= t3 <= NT
    assert len([x for x in open(cache).read().split("\n") if x.strip()]) == 2
    # the picked tune computes the same scores as the default within the bar
    r0 = api.similarity(pa, pa, w.pairs, om, want_match=True)
    r1 = api.similarity(pa, pa, w.pairs, om, want_match=True, tune=t1)
    assert float((r0.scores - r1.scores).abs().max()) <= 2 * ATOL_S


@pytest.mark.parametrize("tune", [183, 228])
def test_deferred_steps_fall_back_without_room(wl, tune):
    """A deferred-steps tune whose workspace has no room for the ranked lists
    (sized as for another tune) matches every pair in the forward instead:
    the same matchings and scores."""
    w, pa, om, ref = wl
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    small = api.ws_size(pa, pa, pairs, B.params(0.8, 40, tune=18))
    assert small < api.ws_size(pa, pa, pairs, B.params(0.8, 40, tune=tune))
    r_def = api.similarity(pa, pa, w.pairs, om, 0.8, 40, want_match=True, tune=tune)
    r_in = api.similarity(pa, pa, w.pairs, om, 0.8, 40, want_match=True, tune=tune, ws_bytes=small)
    assert np.array_equal(r_def.match.cpu().numpy(), r_in.match.cpu().numpy())
    assert np.array_equal(r_def.scores.cpu().numpy(), r_in.scores.cpu().numpy())


def test_deferred_steps_in_captured_graph(wl):
    """The plan and the forward with deferred steps (three kernels) captured
    once and replayed: the same results as the direct call, bit for bit."""
    w, pa, om, ref = wl
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    tune = 183
    d_pairs = torch.from_numpy(pairs).to(DEV)
    ws = api.Workspace(torch.device(DEV))
    nb = api.ws_size(pa, pa, pairs, B.params(0.8, 40, tune=tune))
    x_off, m_off = api.out_offsets(pa, pa, pairs)
    out = {"scores": torch.empty(len(pairs), device=DEV),
           "match": torch.empty(int(m_off[-1]), dtype=torch.int32, device=DEV)}

    def sim(flags):
        api.similarity(pa, pa, pairs, om, 0.8, 40, want_match=True, ws=ws, d_pairs=d_pairs, out=out,
                       check_status=False, flags=flags, ws_bytes=nb, tune=tune)

    sim(0)
    torch.cuda.synchronize()
    s0, m0 = out["scores"].clone(), out["match"].clone()
    g_plan, g_fwd = api.Graph(torch.device(DEV)), api.Graph(torch.device(DEV))
    with g_plan.capture():
        sim(B.CF_FLAG_PLAN_ONLY)
    with g_fwd.capture():
        sim(B.CF_FLAG_REUSE_PLAN)
    for _ in range(3):
        out["scores"].zero_()
        out["match"].fill_(-7)
        g_plan.launch()
        g_fwd.launch()
        torch.cuda.synchronize()
        assert torch.equal(out["scores"], s0) and torch.equal(out["match"], m0)
