"""The C-ABI library on the host: it loads, exports every symbol include/cfsim.h
declares, builds correct CSR packs, and rejects bad input with the documented
status.  No call here touches a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from gen import CFG, config1, config2
from paper_1707_02423_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_1707_02423_gb300 import build

        build.build()
    return B.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "cfsim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(B.SIGNATURES), set(names) ^ set(B.SIGNATURES)
    assert L.cf_abi_version() == 2
    for s in range(7):
        assert L.cf_status_string(s)


def views_of(cfgs, F):
    keep = []
    views = (B.cf_cfg_view * len(cfgs))()
    for k, c in enumerate(cfgs):
        arrs = [np.ascontiguousarray(c.src, np.int32), np.ascontiguousarray(c.dst, np.int32),
                np.ascontiguousarray(c.w, np.float32), np.ascontiguousarray(c.attr, np.float32)]
        keep += arrs
        views[k] = B.cf_cfg_view(c.n, len(c.src), *[a.ctypes.data for a in arrs])
    return views, keep


def build_host(L, cfgs, F):
    views, keep = views_of(cfgs, F)
    n = C.c_size_t(0)
    B.check(L.cf_pack_size(views, len(cfgs), F, C.byref(n)))
    buf = np.zeros(n.value, np.uint8)
    B.check(L.cf_pack_host(views, len(cfgs), F, buf.ctypes.data, n.value))
    return buf


HDR = np.dtype([("magic", "<u4"), ("version", "<u4"), ("n_cfgs", "<i4"), ("F", "<i4"), ("F_pad", "<i4"),
                ("max_blocks", "<i4"), ("max_out", "<i4"), ("max_in", "<i4"), ("n_blocks", "<i8"),
                ("n_edges", "<i8"), ("n_user", "<i8"), ("total", "<i8"), ("off_node", "<i8"), ("off_edge", "<i8"),
                ("off_uedge", "<i8"), ("off_out_ptr", "<i8"), ("off_in_ptr", "<i8"), ("off_out_adj", "<i8"),
                ("off_in_adj", "<i8"), ("off_in_eid", "<i8"), ("off_u2c", "<i8"), ("off_attr", "<i8"),
                ("off_xdeg", "<i8")])


def parse(buf):
    h = np.frombuffer(buf[:HDR.itemsize].tobytes(), HDR)[0]

    def arr(off, dt, n):
        return np.frombuffer(buf[off:off + np.dtype(dt).itemsize * n].tobytes(), dt)

    nb, ne, nu, nc = int(h["n_blocks"]), int(h["n_edges"]), int(h["n_user"]), int(h["n_cfgs"])
    adj = np.dtype([("nbr", "<i4"), ("w", "<f4")])
    return {
        "h": h,
        "node": arr(h["off_node"], "<i4", nc + 1), "edge": arr(h["off_edge"], "<i4", nc + 1),
        "uedge": arr(h["off_uedge"], "<i4", nc + 1),
        "out_ptr": arr(h["off_out_ptr"], "<i4", nb + 1), "in_ptr": arr(h["off_in_ptr"], "<i4", nb + 1),
        "out_adj": arr(h["off_out_adj"], adj, ne), "in_adj": arr(h["off_in_adj"], adj, ne),
        "in_eid": arr(h["off_in_eid"], "<i4", ne), "u2c": arr(h["off_u2c"], "<i4", nu),
        "attr": arr(h["off_attr"], "<f4", nb * int(h["F_pad"])).reshape(nb, int(h["F_pad"])),
        "xdeg": arr(h["off_xdeg"], "<u1", nc),
    }


def test_pack_layout_matches_the_graphs(L):
    cfgs = config2(12).cfgs_a
    # add duplicate edges and a self-loop to one graph
    c0 = cfgs[0]
    cfgs[0] = CFG(c0.n, np.concatenate([c0.src, [c0.src[0], 2]]).astype(np.int32),
                  np.concatenate([c0.dst, [c0.dst[0], 2]]).astype(np.int32),
                  np.concatenate([c0.w, [0.25, 0.5]]).astype(np.float32), c0.attr)
    buf = build_host(L, cfgs, 13)
    P = parse(buf)
    h = P["h"]
    assert h["magic"] == 0x4B504643 and h["F"] == 13 and h["F_pad"] == 16
    assert h["version"] == 2
    for off in ("off_node", "off_out_ptr", "off_out_adj", "off_attr", "off_u2c", "off_xdeg"):
        assert h[off] % 256 == 0
    for c, g in enumerate(cfgs):
        b0, b1 = P["node"][c], P["node"][c + 1]
        assert b1 - b0 == g.n
        # dense weighted adjacency from the pack vs from the edge list (duplicates summed)
        W = np.zeros((g.n, g.n))
        np.add.at(W, (g.src, g.dst), g.w.astype(np.float64))
        Wo = np.zeros_like(W)
        Wi = np.zeros_like(W)
        for i in range(g.n):
            for e in range(P["out_ptr"][b0 + i], P["out_ptr"][b0 + i + 1]):
                Wo[i, P["out_adj"][e]["nbr"]] += P["out_adj"][e]["w"]
            for e in range(P["in_ptr"][b0 + i], P["in_ptr"][b0 + i + 1]):
                Wi[P["in_adj"][e]["nbr"], i] += P["in_adj"][e]["w"]
                assert P["out_adj"][P["in_eid"][e]]["nbr"] == i
        assert np.allclose(Wo, W, atol=1e-6) and np.allclose(Wi, W, atol=1e-6)
        # user edge -> distinct edge
        u0 = P["uedge"][c]
        for e in range(len(g.src)):
            d = P["u2c"][u0 + e]
            assert P["out_adj"][d]["nbr"] == g.dst[e]
            assert P["out_ptr"][b0 + g.src[e]] <= d < P["out_ptr"][b0 + g.src[e] + 1]
        assert np.array_equal(P["attr"][b0:b1, :13], g.attr) and not P["attr"][b0:b1, 13:].any()
        # the per-CFG flag: some block with more than two distinct out- or in-neighbours
        es = set(zip(g.src.tolist(), g.dst.tolist()))
        od = np.bincount([a for a, _ in es], minlength=g.n)
        idg = np.bincount([b for _, b in es], minlength=g.n)
        assert P["xdeg"][c] == int(od.max() > 2 or idg.max() > 2)
    info = B.cf_pack_info()
    B.check(L.cf_pack_info_get(buf.ctypes.data, C.byref(info)))
    assert info.n_cfgs == 12 and info.n_user_edges == sum(len(c.src) for c in cfgs)
    assert info.n_edges == info.n_user_edges - 1  # one duplicate merged


def _status(L, cfgs, F):
    views, keep = views_of(cfgs, F)
    n = C.c_size_t(0)
    return L.cf_pack_size(views, len(cfgs), F, C.byref(n))


def test_pack_validation(L):
    ok = config1().cfgs_a[0]
    assert _status(L, [ok], 13) == 0
    bad_idx = CFG(ok.n, ok.src.copy(), ok.dst.copy(), ok.w, ok.attr)
    bad_idx.dst[0] = ok.n
    assert _status(L, [bad_idx], 13) == 1
    assert b"out of range" in L.cf_last_error_detail()
    bad_w = CFG(ok.n, ok.src, ok.dst, ok.w.copy(), ok.attr)
    bad_w.w[1] = -0.5
    assert _status(L, [bad_w], 13) == 1
    bad_a = CFG(ok.n, ok.src, ok.dst, ok.w, ok.attr.copy())
    bad_a.attr[0, 0] = np.nan
    assert _status(L, [bad_a], 13) == 1
    assert _status(L, [ok], 40) == 3  # F above the supported 32
    empty = CFG(0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros((0, 13), np.float32))
    assert _status(L, [empty], 13) == 1
    single = CFG(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32), np.ones((1, 13), np.float32))
    assert _status(L, [single], 13) == 0


def test_sizes_and_argument_checks(L):
    w = config1()
    buf = build_host(L, w.cfgs_a, 13)
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    xs, ms = C.c_int64(0), C.c_int64(0)
    B.check(L.cf_out_sizes(buf.ctypes.data, buf.ctypes.data, pairs.ctypes.data, len(pairs), C.byref(xs), C.byref(ms)))
    n = np.array([c.n for c in w.cfgs_a])
    assert xs.value == int(sum(n[a] * n[b] for a, b in w.pairs)) and ms.value == int(sum(n[a] for a, _ in w.pairs))
    prm = B.params()
    ws = C.c_size_t(0)
    B.check(L.cf_similarity_ws_size(buf.ctypes.data, buf.ctypes.data, pairs.ctypes.data, len(pairs), C.byref(prm),
                                    C.byref(ws)))
    assert ws.value > 0
    bad = pairs.copy()
    bad[3, 1] = 99
    assert L.cf_out_sizes(buf.ctypes.data, buf.ctypes.data, bad.ctypes.data, len(bad), C.byref(xs), C.byref(ms)) == 1
    # device calls reject bad arguments before touching the device
    dummy = C.c_void_p(1)
    for bad_prm in (B.params(alpha=1.0), B.params(alpha=-0.1), B.params(K=-1), B.params(norm_mode=7),
                    B.params(flags=1 << 5)):
        assert L.cf_similarity(dummy, dummy, dummy, 3, C.byref(bad_prm), dummy, None, None, None, dummy, 1 << 20,
                               None) == 1
    assert L.cf_similarity(None, dummy, dummy, 3, C.byref(prm), dummy, None, None, None, dummy, 1 << 20, None) == 1
    assert L.cf_similarity(dummy, dummy, dummy, 3, C.byref(prm), dummy, None, None, None, dummy, 16, None) == 2
    assert L.cf_topk(dummy, 2, 10, 11, dummy, dummy, None) == 1


def test_graph_and_probe_argument_checks(L):
    h = C.c_void_p(None)
    assert L.cf_graph_begin(None) == 1  # the legacy default stream cannot be captured
    assert L.cf_graph_end(None, C.byref(h)) == 1
    assert L.cf_graph_launch(None, None) == 1
    assert L.cf_graph_nodes(None) == -1
    assert L.cf_graph_destroy(None) == 0
    r = B.cf_probe_result()
    n = C.c_size_t(0)
    assert L.cf_probe_ws_size(7, C.byref(n)) == 1
    assert L.cf_probe(0, None, 0, 1, None, C.byref(r)) == 1


def test_tune_table_and_deferred_steps_room(L):
    """The tune table (host only): 240 distinct configurations, ids 181-240 the
    ones whose matching steps are deferred, and only those tunes size the
    workspace with room for every pair's ranked lists (6 bytes per entry,
    plus the list of deferred pairs)."""
    from paper_1707_02423_gb300 import api

    assert L.cf_num_tunes() == 240
    seen = set()
    for t in range(1, 241):
        d = api.tune_info(t)
        assert (d["matching"] == "ranked, sequential steps in a second kernel") == (t >= 181)
        seen.add((d["threads_per_cta"], d["smallest_group"], d["matching"], d["cluster"]))
    assert len(seen) == 240
    w = config2(12)
    buf = build_host(L, w.cfgs_a, 13)
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    xs, ms = C.c_int64(0), C.c_int64(0)
    B.check(L.cf_out_sizes(buf.ctypes.data, buf.ctypes.data, pairs.ctypes.data, len(pairs), C.byref(xs), C.byref(ms)))

    def ws(tune, flags=0):
        n = C.c_size_t(0)
        B.check(L.cf_similarity_ws_size(buf.ctypes.data, buf.ctypes.data, pairs.ctypes.data, len(pairs),
                                        C.byref(B.params(tune=tune, flags=flags)), C.byref(n)))
        return n.value

    base = ws(18)
    assert ws(0) == base and ws(180) == base
    for t in (181, 198, 228, 240):
        assert ws(t) - base >= 6 * xs.value + 4 * len(pairs)
    # the plain per-pair form runs the steps in place: no extra room
    assert ws(228, B.CF_FLAG_PER_PAIR_LAUNCH) == ws(18, B.CF_FLAG_PER_PAIR_LAUNCH)
