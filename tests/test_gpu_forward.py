"""GPU parity of the forward path (cf_similarity / cf_match / cf_topk) against
the FP64 oracle, through the C ABI.

Bar: X entries and graph scores within max-abs 1e-5; matchings identical
wherever every greedy decision of the oracle wins by more than 1e-6 (else a
valid matching of min(n_a, n_b) pairs); top-k and matching of given matrices
bit-exact."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from _helpers import ATOL_S, ATOL_X, TIE_EPS, eps_greedy, greedy_margin, valid_matching  # noqa: E402
from gen import CFG, config1, config2, config3, config5, structured_cfg  # noqa: E402
from paper_1707_02423_gb300 import _binding as B  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def compare(cfgs_a, cfgs_b, pairs, F, omega=None, alpha=0.8, K=40, per_pair=False, norm_mode=0,
            check_x=True, sample=None, tune=0, flags=0):
    pa = api.Pack(cfgs_a, F, device=DEV)
    pb = pa if cfgs_b is cfgs_a else api.Pack(cfgs_b, F, device=DEV)
    om = np.ones(F) if omega is None else np.asarray(omega, np.float64)
    res = api.similarity(pa, pb, pairs, torch.tensor(om, dtype=torch.float32, device=DEV), alpha, K,
                         want_x=check_x, want_match=True, per_pair=per_pair, norm_mode=norm_mode, tune=tune,
                         flags=flags)
    scores = res.scores.cpu().numpy()
    match = res.match.cpu().numpy()
    X = res.X.cpu().numpy() if check_x else None
    idx = range(len(pairs)) if sample is None else sample
    worst_x = worst_s = 0.0
    exact = tied = 0
    for p in idx:
        a, b = pairs[p]
        A, Bc = cfgs_a[a], cfgs_b[b]
        ref = oracle.similarity(A, Bc, om, alpha, K, normalize=(norm_mode == 0))["X"]
        m_ref, s_ref = oracle.greedy_match(ref)
        got = X[res.x_off[p]:res.x_off[p + 1]].reshape(A.n, Bc.n) if check_x else None
        if check_x:
            worst_x = max(worst_x, float(np.abs(got - ref).max()))
        m = match[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, A.n, Bc.n), (p, m)
        if greedy_margin(ref) > TIE_EPS:
            # every greedy decision is clear: the matching is unique
            assert np.array_equal(m, m_ref), (p, m, m_ref)
            worst_s = max(worst_s, abs(float(scores[p]) - s_ref))
            exact += 1
        else:
            # tied decisions: several matchings are correct; check that this one
            # is greedy within the X tolerance and that its score is its own sum
            tied += 1
            if check_x:
                assert eps_greedy(got, ref, m, 2 * ATOL_X), p
            s_own = sum(ref[i, m[i]] for i in range(A.n) if m[i] >= 0)
            worst_s = max(worst_s, abs(float(scores[p]) - s_own))
    assert worst_x <= ATOL_X, worst_x
    assert worst_s <= ATOL_S, worst_s
    return {"worst_x": worst_x, "worst_s": worst_s, "exact": exact, "tied": tied, "scores": scores,
            "match": match, "X": X, "res": res}


def test_cfg1_all_pairs():
    w = config1()
    r = compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F)
    assert r["exact"] >= 20  # most pairs have clear greedy decisions


def test_cfg2_subset_all_classes():
    # 40 CFGs with n in [8, 120]: warp-, CTA- and global-class pairs
    w = config2(40)
    ns = [c.n for c in w.cfgs_a]
    assert max(ns) * sorted(ns)[-2] > 5632  # at least one global-class pair
    compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F, omega=np.linspace(0.5, 1.5, 13))


def test_per_pair_form_matches_oracle():
    w = config2(14)
    compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F, per_pair=True)


def test_per_pair_form_over_streams_matches_oracle():
    """The plain form with its launches spread over 32 streams: small pairs
    and global-class pairs (each stream with its own scratch slot)."""
    w = config2(14)
    compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F, per_pair=True, flags=B.CF_FLAG_PER_PAIR_STREAMS)
    big = config3(3, 500, 900)
    compare(big.cfgs_a, big.cfgs_a, big.pairs, big.F, per_pair=True, flags=B.CF_FLAG_PER_PAIR_STREAMS)


@pytest.mark.parametrize("alpha,K", [(0.0, 40), (0.5, 7), (0.95, 40), (0.8, 0), (0.8, 1)])
def test_alpha_and_K(alpha, K):
    w = config1()
    compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F, alpha=alpha, K=K)


def test_linear_mode_matches_oracle():
    # CF_NORM_NONE: plain fixed-point iteration of the Table 1 linear system
    w = config1()
    compare(w.cfgs_a, w.cfgs_a, w.pairs[:10], w.F, alpha=0.5, K=60, norm_mode=1)


def edge_case_cfgs():
    rng = np.random.default_rng(123)
    F = 5
    out = []
    # a single block, no edges
    out.append(CFG(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                   rng.uniform(0, 5, (1, F)).astype(np.float32)))
    # complete digraph with self-loops: degrees 7 (register lists overflow)
    n = 7
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    out.append(CFG(n, s.ravel().astype(np.int32), d.ravel().astype(np.int32),
                   rng.dirichlet(np.ones(n * n)).astype(np.float32) * n, rng.uniform(0, 5, (n, F)).astype(np.float32)))
    # duplicate edges and zero-attribute rows
    c = structured_cfg(rng, 12, 3, F - 1)
    attr = c.attr.copy()
    attr[[1, 4]] = 0.0
    out.append(CFG(c.n, np.concatenate([c.src, c.src[:3]]).astype(np.int32),
                   np.concatenate([c.dst, c.dst[:3]]).astype(np.int32),
                   np.concatenate([c.w, c.w[:3]]).astype(np.float32), attr))
    # all-zero attributes: uniform restart term
    c = structured_cfg(rng, 9, 3, F - 1)
    out.append(CFG(c.n, c.src, c.dst, c.w, np.zeros((c.n, F), np.float32)))
    # a chain (n_col = 1 against the single block), a star with in-degree 30
    out.append(structured_cfg(rng, 40, 0, F - 1))
    n = 31
    out.append(CFG(n, np.arange(1, n).astype(np.int32), np.zeros(n - 1, np.int32),
                   np.ones(n - 1, np.float32), rng.uniform(0, 5, (n, F)).astype(np.float32)))
    # a long thin graph (rows >> columns) and a big one for the CTA class
    out.append(structured_cfg(rng, 300, 5, F - 1))
    out.append(structured_cfg(rng, 70, 5, F - 1))
    return out, F


def test_edge_cases_all_pairs_both_orders():
    cfgs, F = edge_case_cfgs()
    n = len(cfgs)
    pairs = np.array([(i, j) for i in range(n) for j in range(n)], np.int32)  # includes (i, i) and both orders
    r = compare(cfgs, cfgs, pairs, F, omega=[1.0, 0.0, 2.0, 0.5, 1.0])
    # S(B, A) = S(A, B)^T
    res, X = r["res"], r["X"]
    for p, (a, b) in enumerate(pairs):
        q = int(b) * n + int(a)
        Xab = X[res.x_off[p]:res.x_off[p + 1]].reshape(cfgs[a].n, cfgs[b].n)
        Xba = X[res.x_off[q]:res.x_off[q + 1]].reshape(cfgs[b].n, cfgs[a].n)
        assert np.abs(Xab - Xba.T).max() <= 2 * ATOL_X


def test_query_shape_f25():
    w = config5(2, 40)
    compare(w.cfgs_a, w.cfgs_b, w.pairs, w.F)


@pytest.mark.parametrize("tune", [0, 1 + 45 * 2, 1 + 45 * 3])  # one CTA per pair; 4- and 8-CTA cluster teams
def test_large_cfgs_global_class(tune):
    w = config3(3, 500, 900)
    compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F, tune=tune)


def test_cfg3_sized_pair_global_tier(capsys):
    """Two of the large-CFG workload's largest CFGs (1,959 x 1,968 blocks:
    X holds 3.9 M entries, the global-memory tier) against the oracle, in
    both orders: X and the score within max-abs 1e-5, the matching exact
    where greedy decisions are clear.  X entries here are about 5e-4, so the
    relative error of X is also bounded and reported beside the max-abs bar."""
    w = config3()
    n = np.array([c.n for c in w.cfgs_a])
    a, b = (int(x) for x in np.argsort(n)[-2:])
    cfgs = [w.cfgs_a[a], w.cfgs_a[b]]
    pairs = np.array([[0, 1], [1, 0]], np.int32)
    pa = api.Pack(cfgs, w.F, device=DEV)
    res = api.similarity(pa, pa, pairs, torch.ones(w.F, device=DEV), 0.8, 40, want_x=True, want_match=True)
    X = res.X.cpu().numpy()
    sc = res.scores.cpu().numpy()
    mt = res.match.cpu().numpy()
    ref = oracle.similarity(cfgs[0], cfgs[1], np.ones(w.F), 0.8, 40)["X"]
    worst_rel = 0.0
    for p, R in ((0, ref), (1, ref.T)):
        got = X[res.x_off[p]:res.x_off[p + 1]].reshape(R.shape)
        err = np.abs(got - R)
        assert err.max() <= ATOL_X, err.max()
        rel = float((err / np.maximum(R, 1e-30)).max())
        worst_rel = max(worst_rel, rel)
        m_ref, s_ref = oracle.greedy_match(R)
        m = mt[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, *R.shape)
        if greedy_margin(R) > TIE_EPS:
            assert np.array_equal(m, m_ref)
            assert abs(float(sc[p]) - s_ref) <= ATOL_S
        else:
            assert eps_greedy(got, R, m, 2 * ATOL_X)
    assert worst_rel <= 1e-3, worst_rel
    with capsys.disabled():
        print(f"\n  1959 x 1968 pair: max-abs error of X within {ATOL_X}, max relative error {worst_rel:.2e}")


def test_full_cfg2_sampled():
    # the bench workload (all 19,900 pairs in one batched call), sampled outputs
    w = config2()
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(w.pairs), 120, replace=False).tolist())
    # include the largest pairs (global class) in the sample
    ns = np.array([c.n for c in w.cfgs_a])
    cost = ns[w.pairs[:, 0]] * ns[w.pairs[:, 1]]
    sample = sorted(set(sample) | set(np.argsort(cost)[-10:].tolist()))
    compare(w.cfgs_a, w.cfgs_a, w.pairs, w.F, sample=sample)


def test_empty_pair_list_is_a_noop():
    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    L = B.lib()
    prm = B.params()
    om = torch.ones(w.F, device=DEV)
    ws = torch.zeros(1 << 16, dtype=torch.uint8, device=DEV)
    B.check(L.cf_similarity(pa.dev.data_ptr(), pa.dev.data_ptr(), ws.data_ptr(), 0, C.byref(prm), om.data_ptr(),
                            None, None, None, ws.data_ptr(), ws.numel(), None))


def _raw_call(pack, pairs_dev, P, om, ws):
    L = B.lib()
    prm = B.params()
    sc = torch.empty(P, device=DEV)
    B.check(L.cf_similarity(pack.dev.data_ptr(), pack.dev.data_ptr(), pairs_dev.data_ptr(), P, C.byref(prm),
                            om.data_ptr(), None, sc.data_ptr(), None, ws.data_ptr(), ws.numel(), None))
    return L.cf_status_check(ws.data_ptr(), None)


def test_device_side_errors_are_reported():
    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    nbytes = api.ws_size(pa, pa, pairs, B.params())
    ws = torch.zeros(nbytes, dtype=torch.uint8, device=DEV)
    om = torch.ones(w.F, device=DEV)
    bad = pairs.copy()
    bad[5, 0] = 1000
    assert _raw_call(pa, torch.from_numpy(bad).to(DEV), len(bad), om, ws) == 1  # CF_ERR_INVALID_ARG
    om_bad = om.clone()
    om_bad[3] = -1.0
    assert _raw_call(pa, torch.from_numpy(pairs).to(DEV), len(pairs), om_bad, ws) == 6  # CF_ERR_NUMERIC
    om_bad[3] = float("nan")
    assert _raw_call(pa, torch.from_numpy(pairs).to(DEV), len(pairs), om_bad, ws) == 6
    # the context is still usable, and a good call clears the status
    assert _raw_call(pa, torch.from_numpy(pairs).to(DEV), len(pairs), om, ws) == 0


def test_workspace_slots_for_pairs_beyond_shared_memory():
    # two 300-block CFGs: their pairs exceed the shared-memory regions and need
    # scratch slots in the workspace
    rng = np.random.default_rng(77)
    cfgs = config2(6).cfgs_a + [structured_cfg(rng, 300, 5, 12), structured_cfg(rng, 290, 5, 12)]
    pairs = np.array([(6, 7), (0, 6), (7, 6), (1, 2)], np.int32)
    pa = api.Pack(cfgs, 13, device=DEV)
    L = B.lib()
    small = C.c_size_t(0)
    B.check(L.cf_similarity_ws_size(pa.host_ptr, pa.host_ptr, np.ascontiguousarray(pairs[3:].repeat(4, 0)).ctypes.data,
                                    4, C.byref(B.params()), C.byref(small)))  # same P, no large pair: fixed part
    om = torch.ones(13, device=DEV)
    d_pairs = torch.from_numpy(pairs).to(DEV)
    ws = torch.zeros(small.value, dtype=torch.uint8, device=DEV)
    assert _raw_call(pa, d_pairs, len(pairs), om, ws) == 2  # CF_ERR_WORKSPACE: no room for a slot
    # exactly one slot: the large pairs share it one after another
    slot = 4 * (3 * 300 * 300 + 2 * 600 + 2 * 300 + 300 + 64 + 64 * 300)  # + per-row busy-column sums
    slot = (slot + 255) // 256 * 256
    ws = torch.zeros(small.value + slot, dtype=torch.uint8, device=DEV)
    sc = torch.empty(len(pairs), device=DEV)
    prm = B.params()
    B.check(L.cf_similarity(pa.dev.data_ptr(), pa.dev.data_ptr(), d_pairs.data_ptr(), len(pairs), C.byref(prm),
                            om.data_ptr(), None, sc.data_ptr(), None, ws.data_ptr(), ws.numel(), None))
    assert L.cf_status_check(ws.data_ptr(), None) == 0
    sc = sc.cpu().numpy()
    for p, (a, b) in enumerate(pairs):
        ref = oracle.similarity(cfgs[a], cfgs[b], np.ones(13))["X"]
        if greedy_margin(ref) > TIE_EPS:
            assert abs(sc[p] - oracle.greedy_match(ref)[1]) <= ATOL_S


def test_match_given_matrices_bit_exact():
    # seeded matrices with many exact ties: the greedy decisions are compared
    # in the same (float32) values on both sides
    rng = np.random.default_rng(42)
    cfgs = [structured_cfg(rng, int(n), 3, 3) for n in (1, 3, 8, 17, 40, 33, 64, 5)]
    pairs = np.array([(i, j) for i in range(len(cfgs)) for j in range(len(cfgs))], np.int32)
    pa = api.Pack(cfgs, 4, device=DEV)
    xs = []
    for a, b in pairs:
        v = rng.integers(0, 6, size=(cfgs[a].n, cfgs[b].n)).astype(np.float32) / 8.0
        xs.append(v.ravel())
    Xh = np.concatenate(xs)
    res = api.match(pa, pa, pairs, torch.from_numpy(Xh).to(DEV))
    mt = res.match.cpu().numpy()
    sc = res.scores.cpu().numpy()
    for p, (a, b) in enumerate(pairs):
        Xp = Xh[res.x_off[p]:res.x_off[p + 1]].reshape(cfgs[a].n, cfgs[b].n).astype(np.float64)
        m_ref, s_ref = oracle.greedy_match(Xp)
        assert np.array_equal(mt[res.m_off[p]:res.m_off[p + 1]], m_ref), p
        assert abs(sc[p] - s_ref) <= 1e-5


def test_topk_exact():
    rng = np.random.default_rng(1)
    Q, Cn, k = 7, 1000, 16
    s = (rng.integers(0, 50, size=(Q, Cn)) / 7.0).astype(np.float32)  # many ties
    top, idx = api.topk(torch.from_numpy(s).to(DEV), k)
    top, idx = top.cpu().numpy(), idx.cpu().numpy()
    for q in range(Q):
        order = np.lexsort((np.arange(Cn), -s[q]))[:k]
        assert np.array_equal(idx[q], order)
        assert np.array_equal(top[q], s[q][order])


def test_cfg_too_large_to_stage():
    # a 4,500-block CFG: its pairs are global-class and its graph does not fit
    # the staging area, so the gather reads the pack directly
    rng = np.random.default_rng(99)
    big = structured_cfg(rng, 4500, 6, 12)
    small = [structured_cfg(rng, n, 3, 12) for n in (5, 9)]
    cfgs = [big] + small
    pairs = np.array([(0, 1), (2, 0), (0, 2)], np.int32)
    compare(cfgs, cfgs, pairs, 13)



def _with_edges(rng, base, n_hubs, fan, n_fans):
    """base with `fan` extra in-edges into each of n_hubs random blocks (hub
    in-degrees about `fan`, like a STOP block reached by many early returns)
    and two extra out-edges from each of n_fans random blocks."""
    src, dst, w = [base.src], [base.dst], [base.w]
    for h in rng.choice(np.arange(1, base.n), n_hubs, replace=False):
        src.append(rng.choice(base.n - 1, fan, replace=False).astype(np.int32))
        dst.append(np.full(fan, h, np.int32))
        w.append(rng.random(fan).astype(np.float32))
    for s in rng.choice(base.n - 1, n_fans, replace=False):
        src.append(np.full(2, s, np.int32))
        dst.append(rng.choice(base.n, 2, replace=False).astype(np.int32))
        w.append(rng.random(2).astype(np.float32))
    return CFG(base.n, np.concatenate(src), np.concatenate(dst), np.concatenate(w), base.attr)


@pytest.mark.parametrize("n_hubs,fan,n_fans", [(2, 30, 0), (0, 0, 48)])
def test_global_tier_busy_columns(n_hubs, fan, n_fans):
    """Global-tier pairs whose column graph has blocks with further
    neighbours: two hubs of in-degree about 30 (their entries go through
    per-row sums of the column lists), or more such blocks than the per-row
    sums hold (their entries are gathered one by one).  700 x 650 blocks:
    X is beyond any cluster's shared memory."""
    rng = np.random.default_rng(1000)
    busy = _with_edges(rng, structured_cfg(rng, 700, 6, 12), n_hubs, fan, n_fans)
    plain = structured_cfg(rng, 650, 6, 12)
    cfgs = [busy, plain]
    pairs = np.array([(1, 0), (0, 1), (0, 0)], np.int32)
    compare(cfgs, cfgs, pairs, 13)
