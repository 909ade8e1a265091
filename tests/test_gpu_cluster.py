"""The cluster tier (pairs too large for one CTA, rows split over the CTAs of
a thread-block cluster, iterates in distributed shared memory) against the
FP64 oracle, for every cluster size the tunes offer, on pairs that span one
CTA's capacity up to beyond an 8-CTA cluster's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from _helpers import ATOL_S, ATOL_X, TIE_EPS, eps_greedy, greedy_margin, valid_matching  # noqa: E402
from gen import CFG, structured_cfg  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


def tune_id(variant, cluster_index, min_level=0, ranked=0):
    """Tune id of (threads variant, smallest-group level, matching policy,
    cluster size index into (0, 2, 4, 8))."""
    return 1 + variant + 3 * min_level + 15 * ranked + 45 * cluster_index


@pytest.fixture(scope="module")
def wl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()
    rng = np.random.default_rng(2024)
    F = 13
    sizes = [150, 190, 230, 260, 330, 420]
    cfgs = []
    for n in sizes:
        c = structured_cfg(rng, n, 6, F - 1)
        cfgs.append(c)
    pairs = np.array([(i, j) for i in range(len(cfgs)) for j in range(len(cfgs)) if i != j], np.int32)
    om = np.linspace(0.7, 1.3, F)
    ref = []
    for a, b in pairs:
        X = oracle.similarity(cfgs[a], cfgs[b], om, 0.8, 40)["X"]
        m, s = oracle.greedy_match(X)
        ref.append((X, m, s, greedy_margin(X) > TIE_EPS))
    pa = api.Pack(cfgs, F, device=DEV)
    return cfgs, pairs, pa, torch.tensor(om, dtype=torch.float32, device=DEV), ref


@pytest.mark.parametrize("variant,ci", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 2)])
def test_cluster_sizes_match_oracle(wl, variant, ci):
    cfgs, pairs, pa, om, ref = wl
    res = api.similarity(pa, pa, pairs, om, 0.8, 40, want_x=True, want_match=True, tune=tune_id(variant, ci))
    X = res.X.cpu().numpy()
    sc = res.scores.cpu().numpy()
    mt = res.match.cpu().numpy()
    worst = 0.0
    for p, (a, b) in enumerate(pairs):
        Xr, m_ref, s_ref, clear = ref[p]
        got = X[res.x_off[p]:res.x_off[p + 1]].reshape(Xr.shape)
        worst = max(worst, float(np.abs(got - Xr).max()))
        m = mt[res.m_off[p]:res.m_off[p + 1]]
        assert valid_matching(m, *Xr.shape), p
        if clear:
            assert np.array_equal(m, m_ref), p
            assert abs(float(sc[p]) - s_ref) <= ATOL_S, p
        else:
            assert eps_greedy(got, Xr, m, 2 * ATOL_X), p
    assert worst <= ATOL_X, worst


def test_cluster_and_global_tiers_agree(wl):
    cfgs, pairs, pa, om, ref = wl
    r0 = api.similarity(pa, pa, pairs, om, want_match=True, tune=tune_id(0, 0))  # global-memory tier
    r1 = api.similarity(pa, pa, pairs, om, want_match=True, tune=tune_id(0, 2))  # 4-CTA clusters
    assert float((r0.scores - r1.scores).abs().max()) <= 2 * ATOL_S


def test_cluster_with_capture_and_noalloc_free_workspace(wl):
    import ctypes as C

    from paper_1707_02423_gb300 import _binding as B

    cfgs, pairs, pa, om, ref = wl
    tune = tune_id(0, 2)
    ws = api.Workspace(DEV)
    prm = B.params(tune=tune)
    nbytes = api.ws_size(pa, pa, pairs, prm)
    out = {"scores": torch.empty(len(pairs), device=DEV)}
    d_pairs = torch.from_numpy(np.ascontiguousarray(pairs)).to(DEV)
    api.similarity(pa, pa, pairs, om, ws=ws, d_pairs=d_pairs, out=out, ws_bytes=nbytes, tune=tune)
    first = out["scores"].clone()
    g = api.Graph(DEV)
    with g.capture():
        api.similarity(pa, pa, pairs, om, ws=ws, d_pairs=d_pairs, out=out, ws_bytes=nbytes, tune=tune,
                       check_status=False)
    out["scores"].zero_()
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out["scores"], first)
    B.check(B.lib().cf_status_check(ws.get(nbytes).data_ptr(), int(torch.cuda.current_stream().cuda_stream)))
