"""GPU parity of the adjoint (cf_similarity_backward) against the FP64 oracle's
reverse-mode gradient (pinned to central finite differences on the CPU).

Bar: max |g - g_ref| <= 1e-4 max |g_ref| over each gradient vector, and
per-element relative 1e-4 for entries at least 1% of the largest.  Only pairs
whose greedy decisions win by more than 1e-5 carry upstream gradient (both
sides then hold the same matching fixed); the others get g = 0."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from _helpers import greedy_margin  # noqa: E402
from gen import config1, config2, config4, config5  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"
REL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def user_offsets(cfgs):
    return np.concatenate([[0], np.cumsum([len(c.src) for c in cfgs])])


def check_close(got, ref, what):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    scale = np.abs(ref).max()
    assert scale > 0, what
    err = np.abs(got - ref)
    assert err.max() <= REL * scale, (what, err.max(), scale)
    big = np.abs(ref) >= 0.01 * scale
    rel = err[big] / np.abs(ref[big])
    assert rel.max() <= REL, (what, rel.max())  # per-element, on entries >= 1% of max
    # every element: relative 1e-4, or absolute 1e-6 of the largest (FP32 sums of many terms)
    assert (err <= np.maximum(REL * np.abs(ref), 1e-6 * scale)).all(), (
        what, float((err / np.maximum(np.abs(ref), 1e-30)).max()), float(err.max() / scale))
    return float(err.max() / scale)


def grad_parity(cfgs_a, cfgs_b, pairs, F, omega, alpha=0.8, K=40, norm_mode=0, seed=0, margin=1e-5, tune=0,
                g_all=None):
    shared = cfgs_b is cfgs_a
    pa = api.Pack(cfgs_a, F, device=DEV)
    pb = pa if shared else api.Pack(cfgs_b, F, device=DEV)
    om = torch.tensor(omega, dtype=torch.float32, device=DEV)
    res = api.similarity(pa, pb, pairs, om, alpha, K, want_match=True, norm_mode=norm_mode)
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.5, 1.5, len(pairs)) if g_all is None else np.full(len(pairs), float(g_all))
    n_used = 0
    ua, ub = user_offsets(cfgs_a), user_offsets(cfgs_b)
    ref_a = np.zeros(ua[-1])
    ref_b = np.zeros(ub[-1]) if not shared else ref_a
    ref_o = np.zeros(F)
    match = res.match.cpu().numpy()
    for p, (a, b) in enumerate(pairs):
        A, Bc = cfgs_a[a], cfgs_b[b]
        X = oracle.similarity(A, Bc, omega, alpha, K, normalize=(norm_mode == 0))["X"]
        if greedy_margin(X) <= margin:
            g[p] = 0.0
            continue
        m_ref, _ = oracle.greedy_match(X)
        assert np.array_equal(match[res.m_off[p]:res.m_off[p + 1]], m_ref), p
        og = oracle.score_gradient(A, Bc, omega, alpha, K, gbar=g[p], match=m_ref, normalize=(norm_mode == 0))
        ref_a[ua[a]:ua[a + 1]] += og["grad_w_a"]
        ref_b[ub[b]:ub[b + 1]] += og["grad_w_b"]
        ref_o += og["grad_omega"]
        n_used += 1
    assert n_used >= max(1, len(pairs) // 3), n_used
    gwa, gwb, gom = api.similarity_backward(pa, pb, pairs, om, res.match,
                                            torch.tensor(g, dtype=torch.float32, device=DEV), alpha, K,
                                            norm_mode=norm_mode, tune=tune)
    check_close(gwa.cpu().numpy(), ref_a, "grad_w_a")
    if not shared:
        check_close(gwb.cpu().numpy(), ref_b, "grad_w_b")
    else:
        assert gwb is None
    check_close(gom.cpu().numpy(), ref_o, "grad_omega")
    return n_used


def test_cfg1_shared_pack():
    w = config1()
    grad_parity(w.cfgs_a, w.cfgs_a, w.pairs, w.F, np.linspace(0.5, 1.5, w.F))


def test_two_packs_f25():
    w = config5(3, 8)
    grad_parity(w.cfgs_a, w.cfgs_b, w.pairs, w.F, np.linspace(1.2, 0.4, w.F), seed=1)


@pytest.mark.parametrize("alpha,K,norm", [(0.5, 10, 1), (0.8, 1, 0), (0.95, 7, 0), (0.8, 50, 0)])
def test_alpha_k_modes(alpha, K, norm):
    w = config1()
    grad_parity(w.cfgs_a, w.cfgs_a, w.pairs[:12], w.F, np.ones(w.F), alpha=alpha, K=K, norm_mode=norm, seed=2)


def test_k0_gradient_is_attribute_term_only():
    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    om = torch.ones(w.F, device=DEV)
    res = api.similarity(pa, pa, w.pairs, om, 0.8, 0, want_match=True)
    g = torch.ones(len(w.pairs), device=DEV)
    gwa, _, gom = api.similarity_backward(pa, pa, w.pairs, om, res.match, g, 0.8, 0)
    assert float(gwa.abs().max()) == 0.0  # K = 0: X = Ehat does not depend on the edges
    assert float(gom.abs().max()) > 0.0


def test_larger_pairs():
    w = config4(6)
    grad_parity(w.cfgs_a, w.cfgs_a, w.pairs, w.F, np.linspace(0.8, 1.2, w.F), seed=3)


def test_autograd_function_matches_oracle():
    w = config2(8)
    pairs = w.pairs[:20]
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    wts = np.concatenate([c.w for c in w.cfgs_a]).astype(np.float32)
    w_a = torch.tensor(wts, device=DEV, requires_grad=True)
    om = torch.ones(w.F, device=DEV, requires_grad=True)
    scores = api.CFSimilarity.apply(w_a, None, om, pa, pa, pairs, 0.8, 40)
    rng = np.random.default_rng(4)
    g = rng.uniform(0.5, 1.5, len(pairs))
    keep = np.array([greedy_margin(oracle.similarity(w.cfgs_a[a], w.cfgs_a[b], np.ones(w.F))["X"]) > 1e-5
                     for a, b in pairs])
    g[~keep] = 0.0
    (scores * torch.tensor(g, dtype=torch.float32, device=DEV)).sum().backward()
    ua = user_offsets(w.cfgs_a)
    ref_a = np.zeros(ua[-1])
    ref_o = np.zeros(w.F)
    for p, (a, b) in enumerate(pairs):
        if not keep[p]:
            continue
        og = oracle.score_gradient(w.cfgs_a[a], w.cfgs_a[b], np.ones(w.F), 0.8, 40, gbar=g[p])
        ref_a[ua[a]:ua[a + 1]] += og["grad_w_a"]
        ref_a[ua[b]:ua[b + 1]] += og["grad_w_b"]
        ref_o += og["grad_omega"]
    check_close(w_a.grad.cpu().numpy(), ref_a, "autograd w")
    check_close(om.grad.cpu().numpy(), ref_o, "autograd omega")


def _largest_and_smallest(w, n_big, n_small):
    n = np.array([c.n for c in w.cfgs_a])
    size = n[w.pairs[:, 0]] * n[w.pairs[:, 1]]
    order = np.argsort(size)
    return w.pairs[np.concatenate([order[-n_big:], order[:n_small]])]


# The adjoint's kernel configurations by tune id (threads per CTA, cluster
# size of the tier for pairs that fit no single CTA): 768/512 threads with no
# cluster tier (those pairs run on one CTA out of L2 slots), then clusters of
# 2, 4 and 8 CTAs (the largest pairs fit only 8-CTA clusters; under 2 and 4
# they too take the L2 tier, now on a whole cluster).
@pytest.mark.parametrize("tune", [3, 2, 48, 93, 92, 138])
def test_tiers_by_tune(tune):
    w = config4()
    pairs = _largest_and_smallest(w, 6, 6)
    grad_parity(w.cfgs_a, w.cfgs_a, pairs, w.F, np.linspace(0.7, 1.3, w.F), seed=5, tune=tune)


def test_cfg4_full_workload():
    """All 256 pairs of the 256-pair gradient workload (n 10-300) in the
    configuration bench.py times (the default), upstream gradient 1 as there."""
    w = config4()
    grad_parity(w.cfgs_a, w.cfgs_a, w.pairs, w.F, np.ones(w.F), g_all=1.0)
