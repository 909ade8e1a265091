"""CUDA-graph capture of a batch step (cf_graph_*) and the on-chip peak probes
(cf_probe) on the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gen import config1, config5  # noqa: E402
from paper_1707_02423_gb300 import _binding as B  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def _setup(w):
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    pb = pa if w.shared else api.Pack(w.cfgs_b, w.F, device=DEV)
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    om = torch.linspace(0.5, 1.5, w.F, device=DEV)
    x_off, m_off = api.out_offsets(pa, pb, pairs)
    out = {"scores": torch.empty(len(pairs), device=DEV),
           "match": torch.empty(int(m_off[-1]), dtype=torch.int32, device=DEV)}
    ws = api.Workspace(DEV)
    ws_bytes = api.ws_size(pa, pb, pairs, B.params())
    ws.get(ws_bytes)
    d_pairs = torch.from_numpy(pairs).to(DEV)
    return pa, pb, pairs, om, out, ws, ws_bytes, d_pairs


def test_captured_step_replays_bit_identical():
    w = config1()
    pa, pb, pairs, om, out, ws, ws_bytes, d_pairs = _setup(w)
    ref = api.similarity(pa, pb, pairs, om, want_match=True)
    g = api.Graph(DEV)
    with g.capture():
        api.similarity(pa, pb, pairs, om, want_match=True, ws=ws, d_pairs=d_pairs, out=out,
                       check_status=False, ws_bytes=ws_bytes)
    assert g.nodes >= 3  # workspace reset, plan kernels, forward
    for _ in range(3):
        out["scores"].fill_(-1.0)
        out["match"].fill_(-7)
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(out["scores"], ref.scores)
        assert torch.equal(out["match"], ref.match)
    B.check(B.lib().cf_status_check(ws.get(ws_bytes).data_ptr(), int(torch.cuda.current_stream().cuda_stream)))


def test_captured_query_step_with_topk():
    w = config5(4, 60)
    pa, pb, pairs, om, out, ws, ws_bytes, d_pairs = _setup(w)
    nq, nc = 4, 60
    ref = api.similarity(pa, pb, pairs, om)
    rt, ri = api.topk(ref.scores.view(nq, nc), 5)
    g = api.Graph(DEV)
    with g.capture():
        api.similarity(pa, pb, pairs, om, ws=ws, d_pairs=d_pairs, out=out, check_status=False, ws_bytes=ws_bytes)
        top, idx = api.topk(out["scores"].view(nq, nc), 5)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(top, rt) and torch.equal(idx, ri)


def test_blocking_call_inside_capture_fails_cleanly():
    w = config1()
    pa, pb, pairs, om, out, ws, ws_bytes, d_pairs = _setup(w)
    api.similarity(pa, pb, pairs, om, ws=ws, d_pairs=d_pairs, out=out, ws_bytes=ws_bytes)
    g = api.Graph(DEV)
    with pytest.raises(B.CfsimError):
        with g.capture():
            api.similarity(pa, pb, pairs, om, ws=ws, d_pairs=d_pairs, out=out, ws_bytes=ws_bytes,
                           check_status=True)  # cf_status_check blocks: not capturable
    torch.cuda.synchronize()
    # the context is still usable
    res = api.similarity(pa, pb, pairs, om)
    assert torch.isfinite(res.scores).all()


@pytest.mark.parametrize("kind,lo,hi", [
    (B.CF_PROBE_SMEM, 32.0, 160.0),   # bytes / clk / SM (128 nominal)
    (B.CF_PROBE_DSMEM, 1.0, 160.0),
    (B.CF_PROBE_FP32, 128.0, 300.0),  # FLOP / clk / SM (256 nominal: 128 FMA lanes)
    (B.CF_PROBE_L2, 4.0, 200.0),
])
def test_probe_is_plausible(kind, lo, hi):
    r = api.probe(kind, reps=2)
    assert r["n_sm"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 200.0 <= r["sm_mhz"] <= 2500.0, r
    assert lo <= r["per_clk_sm"] <= hi, r
    assert abs(r["rate"] - r["work"] / (r["best_ms"] * 1e-3)) <= 1e-6 * r["rate"]
