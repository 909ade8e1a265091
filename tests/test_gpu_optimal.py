"""CF_MATCH_OPTIMAL (maximum-weight assignment, one warp per pair) against
the oracle's assignment (pinned to brute force on tiny matrices).

Bar: the assignment is a valid matching of min(n_a, n_b) pairs whose summed
value, evaluated on the same matrix, is within 1e-5 of the optimum; it is
the oracle's assignment wherever that optimum is unique by more than 1e-5
(checked by re-solving with the oracle's pairs forbidden one at a time on
small cases)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from _helpers import ATOL_S, valid_matching  # noqa: E402
from gen import config1, config2, config5  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def value(X, m):
    return float(sum(X[i, m[i]] for i in range(X.shape[0]) if m[i] >= 0))


def unique_margin(X, m_opt):
    """How much worse the best assignment avoiding one of the optimum's pairs
    is (a lower bound on the optimum's uniqueness margin)."""
    best = oracle.optimal_match(X)[1]
    gap = np.inf
    for i in range(X.shape[0]):
        if m_opt[i] < 0:
            continue
        Y = X.copy()
        Y[i, m_opt[i]] = -1e3
        gap = min(gap, best - oracle.optimal_match(Y)[1])
    return gap


def test_given_matrices_random_and_tied():
    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    rng = np.random.default_rng(7)
    mats = []
    for k, (a, b) in enumerate(w.pairs):
        na, nb = w.cfgs_a[a].n, w.cfgs_a[b].n
        X = rng.random((na, nb)).astype(np.float32)
        if k % 4 == 0:
            X = (np.round(X * 3) / 3).astype(np.float32)  # many ties
        mats.append(X)
    Xd = torch.from_numpy(np.concatenate([m.ravel() for m in mats])).to(DEV)
    res = api.match(pa, pa, w.pairs, Xd, optimal=True)
    sc = res.scores.cpu().numpy()
    mt = res.match.cpu().numpy()
    exact = 0
    for p, (a, b) in enumerate(w.pairs):
        X = mats[p].astype(np.float64)
        m = mt[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, *X.shape), p
        m_ref, s_ref = oracle.optimal_match(X)
        assert abs(value(X, m) - s_ref) <= 1e-5, (p, value(X, m), s_ref)
        assert abs(float(sc[p]) - value(X, m)) <= 1e-5, p
        if p % 4 != 0 and unique_margin(X, m_ref) > 1e-5:
            assert np.array_equal(m, m_ref), p
            exact += 1
    assert exact >= 10


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (33, 5), (5, 33), (70, 70), (130, 64)])
def test_shapes_including_transposed(shape):
    from gen import CFG

    rng = np.random.default_rng(sum(shape))
    F = 3
    cfgs = [CFG(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                rng.uniform(0, 1, (n, F)).astype(np.float32)) for n in shape]
    pa = api.Pack(cfgs, F, device=DEV)
    X = rng.random(shape).astype(np.float32)
    res = api.match(pa, pa, [(0, 1)], torch.from_numpy(X.ravel()).to(DEV), optimal=True)
    m = res.match.cpu().numpy()
    assert valid_matching(m, *shape)
    _, s_ref = oracle.optimal_match(X.astype(np.float64))
    assert abs(value(X.astype(np.float64), m) - s_ref) <= 1e-5


def test_many_pairs_through_the_slot_pool():
    """A batch large enough that every CTA's shared-memory slot pool fills,
    fragments and turns over many times, with pairs of every width up to 128
    blocks (the register form's limit, including 32/33, 64/65, 96/97 and
    127/128), on near-rank-one matrices like X_K."""
    from gen import CFG

    rng = np.random.default_rng(5)
    F = 2
    sizes = np.concatenate([[1, 2, 31, 32, 33, 64, 65, 96, 97, 127, 128], rng.integers(1, 129, 49)])
    cfgs = [CFG(int(n), np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                np.ones((int(n), F), np.float32)) for n in sizes]
    pairs = np.array([(a, b) for a in range(len(cfgs)) for b in range(len(cfgs))], np.int32)
    pairs = pairs[rng.permutation(len(pairs))[:2500]]
    mats = []
    for a, b in pairs:
        na, nb = int(sizes[a]), int(sizes[b])
        X = np.outer(rng.uniform(0.5, 1, na), rng.uniform(0.5, 1, nb)) + 0.02 * rng.random((na, nb))
        mats.append(X.astype(np.float32))
    pa = api.Pack(cfgs, F, device=DEV)
    res = api.match(pa, pa, pairs, torch.from_numpy(np.concatenate([m.ravel() for m in mats])).to(DEV), optimal=True)
    sc, mt = res.scores.cpu().numpy(), res.match.cpu().numpy()
    for p in range(len(pairs)):
        X = mats[p].astype(np.float64)
        m = mt[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, *X.shape), p
        _, s_ref = oracle.optimal_match(X)
        tol = 1e-5 + 1e-6 * min(X.shape)
        assert abs(value(X, m) - s_ref) <= tol, (p, X.shape, value(X, m), s_ref)
        assert abs(float(sc[p]) - value(X, m)) <= tol, p


def test_unstaged_path_matches_the_oracle():
    """The register form with every matrix read from global memory: the path
    a warp takes when its bounded wait for shared-memory slots runs out
    (forced for every pair by CF_FLAG_OPT_UNSTAGED), on near-rank-one
    matrices of every width up to 128, against the oracle's optimum and the
    staged path's assignment value."""
    from gen import CFG

    from paper_1707_02423_gb300 import _binding as B

    rng = np.random.default_rng(11)
    F = 2
    sizes = np.concatenate([[1, 2, 31, 32, 33, 64, 65, 127, 128], rng.integers(1, 129, 21)])
    cfgs = [CFG(int(n), np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                np.ones((int(n), F), np.float32)) for n in sizes]
    pairs = np.array([(a, b) for a in range(len(cfgs)) for b in range(len(cfgs))], np.int32)
    pairs = pairs[rng.permutation(len(pairs))[:400]]
    mats = []
    for a, b in pairs:
        na, nb = int(sizes[a]), int(sizes[b])
        X = np.outer(rng.uniform(0.5, 1, na), rng.uniform(0.5, 1, nb)) + 0.02 * rng.random((na, nb))
        mats.append(X.astype(np.float32))
    pa = api.Pack(cfgs, F, device=DEV)
    Xd = torch.from_numpy(np.concatenate([m.ravel() for m in mats])).to(DEV)
    un = api.match(pa, pa, pairs, Xd, optimal=True, flags=B.CF_FLAG_OPT_UNSTAGED)
    st = api.match(pa, pa, pairs, Xd, optimal=True)
    su, mu = un.scores.cpu().numpy(), un.match.cpu().numpy()
    ss = st.scores.cpu().numpy()
    for p in range(len(pairs)):
        X = mats[p].astype(np.float64)
        m = mu[un.m_off[p]:un.m_off[p + 1]]
        assert valid_matching(m, *X.shape), p
        _, s_ref = oracle.optimal_match(X)
        tol = 1e-5 + 1e-6 * min(X.shape)
        assert abs(value(X, m) - s_ref) <= tol, (p, X.shape, value(X, m), s_ref)
        assert abs(float(su[p]) - float(ss[p])) <= tol, p


def test_nan_row_sets_numeric_status():
    from gen import CFG

    from paper_1707_02423_gb300 import _binding as B

    F = 2
    cfgs = [CFG(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                np.ones((n, F), np.float32)) for n in (6, 9)]
    X = np.random.default_rng(3).random((6, 9)).astype(np.float32)
    X[4, :] = np.nan
    pa = api.Pack(cfgs, F, device=DEV)
    with pytest.raises(B.CfsimError) as e:
        api.match(pa, pa, [(0, 1)], torch.from_numpy(X.ravel()).to(DEV), optimal=True)
    assert e.value.status == 6


def test_similarity_with_optimal_matching_cfg2_subset():
    w = config2(16)
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    om = torch.ones(w.F, device=DEV)
    res = api.similarity(pa, pa, w.pairs, om, want_match=True, optimal=True)
    greedy = api.similarity(pa, pa, w.pairs, om, want_match=True)
    sc, mt = res.scores.cpu().numpy(), res.match.cpu().numpy()
    gs = greedy.scores.cpu().numpy()
    for p, (a, b) in enumerate(w.pairs):
        X = oracle.similarity(w.cfgs_a[a], w.cfgs_a[b], np.ones(w.F))["X"]
        m = mt[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, *X.shape), p
        _, s_ref = oracle.optimal_match(X)
        assert abs(value(X, m) - s_ref) <= 2 * ATOL_S, p
        assert abs(float(sc[p]) - s_ref) <= 2 * ATOL_S, p
        assert float(sc[p]) >= float(gs[p]) - 2 * ATOL_S  # the optimum is never below greedy


def test_optimal_query_shapes_two_packs():
    w = config5(2, 40)
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    pb = api.Pack(w.cfgs_b, w.F, device=DEV)
    om = torch.ones(w.F, device=DEV)
    res = api.similarity(pa, pb, w.pairs, om, want_match=True, optimal=True)
    sc = res.scores.cpu().numpy()
    for p in range(0, len(w.pairs), 7):
        a, b = w.pairs[p]
        X = oracle.similarity(w.cfgs_a[a], w.cfgs_b[b], np.ones(w.F))["X"]
        _, s_ref = oracle.optimal_match(X)
        assert abs(float(sc[p]) - s_ref) <= 2 * ATOL_S, p


def test_optimal_needs_x():
    import ctypes as C

    from paper_1707_02423_gb300 import _binding as B

    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    d_pairs = torch.from_numpy(pairs).to(DEV)
    prm = B.params(match_mode=B.CF_MATCH_OPTIMAL)
    n = api.ws_size(pa, pa, pairs, prm)
    ws = torch.empty(n, dtype=torch.uint8, device=DEV)
    sc = torch.empty(len(pairs), device=DEV)
    om = torch.ones(w.F, device=DEV)
    st = B.lib().cf_similarity(pa.dev.data_ptr(), pa.dev.data_ptr(), d_pairs.data_ptr(), len(pairs), C.byref(prm),
                               om.data_ptr(), None, sc.data_ptr(), None, ws.data_ptr(), n, None)
    assert st == 1  # CF_ERR_INVALID_ARG: d_X is required
