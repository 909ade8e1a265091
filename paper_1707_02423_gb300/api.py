"""Python API over the C ABI: packs, workspaces, and the similarity calls.

PyTorch supplies device memory and streams only; every step of the path runs
in libcfsim.so's kernels.  Tensors passed in must live on the current CUDA
device.
"""
from __future__ import annotations

import contextlib
import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _binding as B


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


class Pack:
    """A CSR batch pack of CFGs (include/cfsim.h, "a1").

    ``cfgs`` is a sequence of objects with ``n``, ``src``, ``dst``, ``w`` and
    ``attr`` ([n, F]).  Keeps the host bytes (for sizing queries) and a device
    copy made by ``cf_pack_cfgs``."""

    def __init__(self, cfgs, F: int, device="cuda"):
        L = B.lib()
        self.F = int(F)
        self.n_blocks = np.array([int(c.n) for c in cfgs], dtype=np.int64)
        self.n_user_edges = np.array([int(len(c.src)) for c in cfgs], dtype=np.int64)
        keep = []
        views = (B.cf_cfg_view * len(cfgs))()
        for k, c in enumerate(cfgs):
            src = np.ascontiguousarray(c.src, dtype=np.int32)
            dst = np.ascontiguousarray(c.dst, dtype=np.int32)
            w = np.ascontiguousarray(c.w, dtype=np.float32)
            attr = np.ascontiguousarray(c.attr, dtype=np.float32)
            if attr.shape != (int(c.n), self.F):
                raise ValueError(f"cfg {k}: attr shape {attr.shape} != ({c.n}, {self.F})")
            keep += [src, dst, w, attr]
            views[k] = B.cf_cfg_view(int(c.n), int(src.size), src.ctypes.data, dst.ctypes.data, w.ctypes.data,
                                     attr.ctypes.data)
        self._views, self._keep = views, keep
        nbytes = C.c_size_t(0)
        B.check(L.cf_pack_size(views, len(cfgs), self.F, C.byref(nbytes)))
        self.host = np.zeros(nbytes.value, dtype=np.uint8)
        B.check(L.cf_pack_host(views, len(cfgs), self.F, self.host.ctypes.data, nbytes.value))
        info = B.cf_pack_info()
        B.check(L.cf_pack_info_get(self.host.ctypes.data, C.byref(info)))
        self.info = info
        self.n_cfgs = info.n_cfgs
        self.dev = None
        if device is not None:
            self.dev = torch.empty(nbytes.value, dtype=torch.uint8, device=device)
            B.check(L.cf_pack_cfgs(views, len(cfgs), self.F, self.dev.data_ptr(), nbytes.value,
                                   _stream_ptr(None)))
        self._keep = None  # the host pack is self-contained

    @property
    def host_ptr(self) -> int:
        return self.host.ctypes.data

    def set_weights(self, w_user: torch.Tensor, stream=None) -> None:
        """Replace the edge weights (user edge order, float32 on the device)."""
        w = w_user.detach().to(torch.float32).contiguous()
        if w.numel() != int(self.info.n_user_edges):
            raise ValueError("w_user has the wrong length")
        B.check(B.lib().cf_pack_set_weights(self.dev.data_ptr(), self.host_ptr, w.data_ptr(), _stream_ptr(stream)))


def out_offsets(pa: Pack, pb: Pack, pairs: np.ndarray):
    """Host copies of x_off and m_off (length P + 1) for a pair list."""
    pairs = np.asarray(pairs, dtype=np.int64)
    na = pa.n_blocks[pairs[:, 0]]
    nb = pb.n_blocks[pairs[:, 1]]
    x_off = np.concatenate([[0], np.cumsum(na * nb)])
    m_off = np.concatenate([[0], np.cumsum(na)])
    return x_off, m_off


class Workspace:
    """A reusable device workspace; grows to the largest size asked for."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        return self.buf


@dataclass
class Result:
    scores: torch.Tensor | None
    match: torch.Tensor | None
    X: torch.Tensor | None
    x_off: np.ndarray
    m_off: np.ndarray

    def X_of(self, p: int, na: int, nb: int) -> torch.Tensor:
        return self.X[int(self.x_off[p]):int(self.x_off[p + 1])].view(na, nb)


def _pairs_np(pairs) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    return p


def ws_size(pa: Pack, pb: Pack, pairs_np: np.ndarray, prm: B.cf_params) -> int:
    n = C.c_size_t(0)
    B.check(B.lib().cf_similarity_ws_size(pa.host_ptr, pb.host_ptr, pairs_np.ctypes.data, len(pairs_np),
                                          C.byref(prm), C.byref(n)))
    return n.value


def similarity(pa: Pack, pb: Pack, pairs, omega: torch.Tensor, alpha: float = 0.8, K: int = 40, *,
               want_x: bool = False, want_scores: bool = True, want_match: bool = False, per_pair: bool = False,
               norm_mode: int = B.CF_NORM_FROB, ws: Workspace | None = None, d_pairs: torch.Tensor | None = None,
               out: dict | None = None, stream=None, check_status: bool = True, flags: int = 0,
               ws_bytes: int | None = None, tune: int = 0, optimal: bool = False) -> Result:
    """X_K, graph scores and greedy matchings for every pair (cf_similarity).

    ``pairs``: int [P, 2] host array of (CFG of pa, CFG of pb).  ``omega``: float32
    [F] on the device.  ``out`` may hold preallocated ``scores`` / ``match`` /
    ``X`` tensors (reused across calls, e.g. under CUDA-graph capture)."""
    L = B.lib()
    pairs_np = _pairs_np(pairs)
    P = len(pairs_np)
    dev = pa.dev.device
    prm = B.params(alpha, K, norm_mode, (B.CF_FLAG_PER_PAIR_LAUNCH if per_pair else 0) | flags, tune,
                   B.CF_MATCH_OPTIMAL if optimal else B.CF_MATCH_GREEDY)
    want_x = want_x or (optimal and (want_scores or want_match))  # the assignment runs on X
    x_off, m_off = out_offsets(pa, pb, pairs_np)
    out = {} if out is None else out
    scores = out.get("scores") if want_scores else None
    if want_scores and scores is None:
        scores = torch.empty(P, dtype=torch.float32, device=dev)
    match = out.get("match") if want_match else None
    if want_match and match is None:
        match = torch.empty(int(m_off[-1]), dtype=torch.int32, device=dev)
    X = out.get("X") if want_x else None
    if want_x and X is None:
        X = torch.empty(int(x_off[-1]), dtype=torch.float32, device=dev)
    if d_pairs is None:
        d_pairs = torch.from_numpy(pairs_np).to(dev)
    ws = ws or Workspace(dev)
    nbytes = ws_size(pa, pb, pairs_np, prm) if ws_bytes is None else ws_bytes
    wbuf = ws.get(nbytes)
    omega = omega.contiguous()
    st = _stream_ptr(stream)
    B.check(L.cf_similarity(pa.dev.data_ptr(), pb.dev.data_ptr(), d_pairs.data_ptr(), P, C.byref(prm),
                            omega.data_ptr(), _ptr(X), _ptr(scores), _ptr(match), wbuf.data_ptr(), wbuf.numel(), st))
    if check_status:
        B.check(L.cf_status_check(wbuf.data_ptr(), st))
    return Result(scores, match, X, x_off, m_off)


def autotune(pa: Pack, pb: Pack, pairs, omega: torch.Tensor, alpha: float = 0.8, K: int = 40, *,
             norm_mode: int = B.CF_NORM_FROB, cache_path: str | None = None, stream=None):
    """The fastest kernel configuration for this workload (cf_autotune):
    returns ``(tune, ms)``; pass ``tune`` to ``similarity``."""
    L = B.lib()
    pairs_np = _pairs_np(pairs)
    prm = B.params(alpha, K, norm_mode)
    n = C.c_size_t(0)
    B.check(L.cf_autotune_ws_size(pa.host_ptr, pb.host_ptr, pairs_np.ctypes.data, len(pairs_np), C.byref(prm),
                                  C.byref(n)))
    ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=pa.dev.device)
    t = C.c_int32(0)
    ms = C.c_float(0.0)
    B.check(L.cf_autotune(pa.host_ptr, pb.host_ptr, pa.dev.data_ptr(), pb.dev.data_ptr(), pairs_np.ctypes.data,
                          len(pairs_np), C.byref(prm), omega.contiguous().data_ptr(), ws.data_ptr(), ws.numel(),
                          cache_path.encode() if cache_path else None, _stream_ptr(stream), C.byref(t), C.byref(ms)))
    return int(t.value), float(ms.value)


def tune_info(tune: int) -> dict:
    r = B.cf_tune_info()
    B.check(B.lib().cf_tune_describe(int(tune), C.byref(r)))
    return {"tune": r.tune, "threads_per_cta": r.threads_per_cta, "smallest_group": r.smallest_group,
            "matching": ("ranked", "ranked in groups of at most a quarter CTA", "rescans",
                         "ranked, sequential steps in a second kernel")[r.matching], "cluster": r.cluster}


def match(pa: Pack, pb: Pack, pairs, X: torch.Tensor, *, ws: Workspace | None = None, stream=None,
          optimal: bool = False, flags: int = 0) -> Result:
    """Greedy (or, with ``optimal``, maximum-weight) matching and scores of
    caller-given matrices (cf_match with X)."""
    L = B.lib()
    pairs_np = _pairs_np(pairs)
    P = len(pairs_np)
    dev = pa.dev.device
    x_off, m_off = out_offsets(pa, pb, pairs_np)
    scores = torch.empty(P, dtype=torch.float32, device=dev)
    mt = torch.empty(int(m_off[-1]), dtype=torch.int32, device=dev)
    d_pairs = torch.from_numpy(pairs_np).to(dev)
    ws = ws or Workspace(dev)
    prm = B.params(match_mode=B.CF_MATCH_OPTIMAL if optimal else B.CF_MATCH_GREEDY, flags=flags)
    wbuf = ws.get(ws_size(pa, pb, pairs_np, prm))
    X = X.contiguous()
    st = _stream_ptr(stream)
    B.check(L.cf_match(pa.dev.data_ptr(), pb.dev.data_ptr(), d_pairs.data_ptr(), P, C.byref(prm), None, X.data_ptr(),
                       mt.data_ptr(), scores.data_ptr(), wbuf.data_ptr(), wbuf.numel(), st))
    B.check(L.cf_status_check(wbuf.data_ptr(), st))
    return Result(scores, mt, X, x_off, m_off)


def distances(pa: Pack, pb: Pack, pairs, p: float = 3.0, *, scale01: bool = False, d_pairs=None,
              out: torch.Tensor | None = None, stream=None, check_status: bool = True) -> torch.Tensor:
    """The five Table 1 distances (Euclidean, Manhattan, Minkowski(p), Jaccard,
    Cosine) of the resized transition matrices of every pair (cf_distances):
    float32 [P, 5], min-max scaled to [0, 1] over the pairs with ``scale01``."""
    L = B.lib()
    pairs_np = _pairs_np(pairs)
    P = len(pairs_np)
    dev = pa.dev.device
    if d_pairs is None:
        d_pairs = torch.from_numpy(pairs_np).to(dev)
    if out is None:
        out = torch.empty(P, 5, dtype=torch.float32, device=dev)
    n = C.c_size_t(0)
    B.check(L.cf_distances_ws_size(P, C.byref(n)))
    ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
    st = _stream_ptr(stream)
    B.check(L.cf_distances(pa.dev.data_ptr(), pb.dev.data_ptr(), d_pairs.data_ptr(), P, float(p),
                           B.CF_DIST_SCALE01 if scale01 else 0, out.data_ptr(), ws.data_ptr(), ws.numel(), st))
    if check_status:
        B.check(L.cf_status_check(ws.data_ptr(), st))
    return out


def score_matrix(pairs, scores: torch.Tensor, n_rows: int, n_cols: int | None = None, *, symmetric: bool = True,
                 d_pairs=None, stream=None) -> torch.Tensor:
    """Dense [n_rows, n_cols] matrix of pair scores (cf_score_matrix)."""
    L = B.lib()
    pairs_np = _pairs_np(pairs)
    dev = scores.device
    n_cols = n_rows if n_cols is None else n_cols
    if d_pairs is None:
        d_pairs = torch.from_numpy(pairs_np).to(dev)
    S = torch.empty(n_rows, n_cols, dtype=torch.float32, device=dev)
    status = torch.empty(1, dtype=torch.int32, device=dev)
    B.check(L.cf_score_matrix(d_pairs.data_ptr(), scores.contiguous().data_ptr(), len(pairs_np), n_rows, n_cols,
                              int(symmetric), S.data_ptr(), status.data_ptr(), _stream_ptr(stream)))
    bad = int(status.item())
    if bad:
        raise B.CfsimError(1, f"pair {bad - 1} is out of range")
    return S


def ward(points: torch.Tensor, stream=None):
    """Ward linkage of the rows of ``points`` [n, dim] (cf_ward): returns
    ``(merge [n-1, 2] int32, height [n-1] float32, size [n-1] int32)`` in
    scipy's linkage convention."""
    L = B.lib()
    X = points.detach().to(torch.float32).contiguous()
    n, dim = X.shape
    dev = X.device
    nb = C.c_size_t(0)
    B.check(L.cf_ward_ws_size(n, C.byref(nb)))
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device=dev)
    merge = torch.empty(max(n - 1, 0), 2, dtype=torch.int32, device=dev)
    height = torch.empty(max(n - 1, 0), dtype=torch.float32, device=dev)
    size = torch.empty(max(n - 1, 0), dtype=torch.int32, device=dev)
    st = _stream_ptr(stream)
    B.check(L.cf_ward(X.data_ptr(), n, dim, merge.data_ptr(), height.data_ptr(), size.data_ptr(), ws.data_ptr(),
                      ws.numel(), st))
    B.check(L.cf_status_check(ws.data_ptr(), st))
    return merge, height, size


def topk_pairs(idx: torch.Tensor, rows: torch.Tensor | None = None, *, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """The winners' pair list of a top-k on the device (cf_topk_pairs):
    int32 [Q k, 2] with (rows[q] or q, idx[q, r]) for every query q and rank r."""
    idx = idx.contiguous()
    Q, k = idx.shape
    if out is None:
        out = torch.empty(Q * k, 2, dtype=torch.int32, device=idx.device)
    B.check(B.lib().cf_topk_pairs(idx.data_ptr(), Q, k, _ptr(rows), out.data_ptr(), _stream_ptr(stream)))
    return out


def ws_size_any(pa: Pack, pb: Pack, P: int, prm: B.cf_params | None = None) -> int:
    """Workspace bytes for any P pairs of these packs (cf_similarity_ws_size_any)."""
    n = C.c_size_t(0)
    B.check(B.lib().cf_similarity_ws_size_any(pa.host_ptr, pb.host_ptr, int(P), C.byref(prm) if prm else None,
                                              C.byref(n)))
    return n.value


def similarity_dev(pa: Pack, pb: Pack, d_pairs: torch.Tensor, omega: torch.Tensor, alpha: float = 0.8, K: int = 40,
                   *, scores: torch.Tensor | None = None, match: torch.Tensor | None = None, ws: Workspace,
                   ws_bytes: int, tune: int = 0, stream=None) -> None:
    """cf_similarity on a pair list that lives only on the device (int32
    [P, 2], e.g. from topk_pairs): scores and / or matchings into the given
    tensors (match needs sum of n_a over the pairs entries; its offsets are
    the prefix sums of n_a in pair order).  Nothing is read back and no
    status is checked, so the call can be captured in a CUDA graph."""
    P = int(d_pairs.shape[0])
    prm = B.params(alpha, K, tune=tune)
    wbuf = ws.get(ws_bytes)
    B.check(B.lib().cf_similarity(pa.dev.data_ptr(), pb.dev.data_ptr(), d_pairs.data_ptr(), P, C.byref(prm),
                                  omega.contiguous().data_ptr(), None, _ptr(scores), _ptr(match), wbuf.data_ptr(),
                                  ws_bytes, _stream_ptr(stream)))


def topk(scores: torch.Tensor, k: int, stream=None, out: tuple | None = None):
    """Per-row top-k of a [Q, C] float32 score matrix: (values, column indices)."""
    s = scores.contiguous()
    Q, Cn = s.shape
    if out is not None:
        top, idx = out
    else:
        top = torch.empty(Q, k, dtype=torch.float32, device=s.device)
        idx = torch.empty(Q, k, dtype=torch.int32, device=s.device)
    B.check(B.lib().cf_topk(s.data_ptr(), Q, Cn, k, top.data_ptr(), idx.data_ptr(), _stream_ptr(stream)))
    return top, idx


def backward_ws_size(pa: Pack, pb: Pack, pairs_np: np.ndarray, prm: B.cf_params) -> int:
    n = C.c_size_t(0)
    B.check(B.lib().cf_similarity_backward_ws_size(pa.host_ptr, pb.host_ptr, pairs_np.ctypes.data, len(pairs_np),
                                                   C.byref(prm), C.byref(n)))
    return n.value


def similarity_backward(pa: Pack, pb: Pack, pairs, omega: torch.Tensor, match: torch.Tensor,
                        grad_scores: torch.Tensor, alpha: float = 0.8, K: int = 40, *,
                        norm_mode: int = B.CF_NORM_FROB, ws: Workspace | None = None, stream=None,
                        tune: int = 0, check_status: bool = True, out: dict | None = None,
                        d_pairs: torch.Tensor | None = None):
    """Gradients of sum_p grad_scores[p] * s_p (cf_similarity_backward) with the
    matching ``match`` (from the forward) held fixed.

    Returns ``(grad_w_a, grad_w_b, grad_omega)``: user-edge-order gradients of
    pack A's and pack B's edge weights (``grad_w_b`` is None when both sides
    are the same pack: everything is in ``grad_w_a``) and of omega.

    ``tune`` selects the adjoint's kernel configuration (0: its default;
    otherwise a tune id's thread count and cluster size).  ``out`` may hold
    zeroed ``grad_w_a`` / ``grad_w_b`` / ``grad_omega`` tensors to accumulate
    into (for CUDA-graph capture, with ``d_pairs``, a sized ``ws`` and
    ``check_status=False``)."""
    L = B.lib()
    pairs_np = _pairs_np(pairs)
    P = len(pairs_np)
    dev = pa.dev.device
    prm = B.params(alpha, K, norm_mode, tune=tune)
    out = {} if out is None else out
    gwa = out.get("grad_w_a")
    if gwa is None:
        gwa = torch.zeros(int(pa.info.n_user_edges), dtype=torch.float32, device=dev)
    gwb = None if pb is pa else out.get("grad_w_b")
    if gwb is None and pb is not pa:
        gwb = torch.zeros(int(pb.info.n_user_edges), dtype=torch.float32, device=dev)
    gom = out.get("grad_omega")
    if gom is None:
        gom = torch.zeros(pa.F, dtype=torch.float32, device=dev)
    ws = ws or Workspace(dev)
    wbuf = ws.get(backward_ws_size(pa, pb, pairs_np, prm))
    if d_pairs is None:
        d_pairs = torch.from_numpy(pairs_np).to(dev)
    g = grad_scores.detach().to(torch.float32).contiguous()
    st = _stream_ptr(stream)
    B.check(L.cf_similarity_backward(pa.dev.data_ptr(), pb.dev.data_ptr(), d_pairs.data_ptr(), P, C.byref(prm),
                                     omega.detach().contiguous().data_ptr(), match.data_ptr(), g.data_ptr(),
                                     gwa.data_ptr(), _ptr(gwb), gom.data_ptr(), wbuf.data_ptr(), wbuf.numel(), st))
    if check_status:
        B.check(L.cf_status_check(wbuf.data_ptr(), st))
    return gwa, gwb, gom


class CFSimilarity(torch.autograd.Function):
    """Graph scores of all pairs as a differentiable function of the edge
    weights (user edge order) and omega; the matching is held fixed in the
    backward pass (it is piecewise constant in the inputs).

    ``apply(w_a, w_b, omega, pack_a, pack_b, pairs, alpha, K)``; pass
    ``w_b = None`` when both sides are the same pack."""

    @staticmethod
    def forward(ctx, w_a, w_b, omega, pack_a, pack_b, pairs, alpha=0.8, K=40):
        pack_a.set_weights(w_a)
        if pack_b is not pack_a:
            pack_b.set_weights(w_b)
        res = similarity(pack_a, pack_b, pairs, omega.detach(), alpha, K, want_match=True)
        ctx.pack_a, ctx.pack_b, ctx.pairs, ctx.alpha, ctx.K = pack_a, pack_b, pairs, alpha, K
        ctx.save_for_backward(omega.detach(), res.match)
        return res.scores

    @staticmethod
    def backward(ctx, g):
        omega, match = ctx.saved_tensors
        ga, gb, go = similarity_backward(ctx.pack_a, ctx.pack_b, ctx.pairs, omega, match, g, ctx.alpha, ctx.K)
        return ga, gb, go, None, None, None, None, None


class Graph:
    """A CUDA graph of cfsim calls (cf_graph_begin / cf_graph_end), replayed
    with ``launch()``.

    Capture runs on the graph's own stream::

        g = Graph()
        with g.capture():
            similarity(..., d_pairs=..., out=..., ws=..., ws_bytes=..., check_status=False)
        g.launch()

    Everything the captured calls touch must already be allocated (pass
    ``d_pairs``, ``out``, a sized ``ws`` and ``ws_bytes``), nothing in the
    capture may block (``check_status=False``), and each kind of call must
    have run once uncaptured before."""

    def __init__(self, device="cuda"):
        self.stream = torch.cuda.Stream(device=device)
        self.handle = None

    @contextlib.contextmanager
    def capture(self):
        L = B.lib()
        if self.handle is not None:
            raise RuntimeError("graph already captured")
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        sp = int(self.stream.cuda_stream)
        with torch.cuda.stream(self.stream):
            B.check(L.cf_graph_begin(sp))
            h = C.c_void_p(None)
            try:
                yield self
            finally:
                st = L.cf_graph_end(sp, C.byref(h))
        B.check(st)
        self.handle = h
        cur.wait_stream(self.stream)

    @property
    def nodes(self) -> int:
        return int(B.lib().cf_graph_nodes(self.handle))

    def launch(self, stream=None) -> None:
        B.check(B.lib().cf_graph_launch(self.handle, _stream_ptr(stream)))

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            try:
                B.lib().cf_graph_destroy(self.handle)
            except Exception:  # interpreter shutdown
                pass
            self.handle = None


def probe(kind: int, reps: int = 3, stream=None) -> dict:
    """On-chip peak of one kind (cf_probe): CF_PROBE_SMEM / L2 / DSMEM (bytes/s)
    or CF_PROBE_FP32 (FLOP/s), with the SM clock of the fastest launch."""
    L = B.lib()
    n = C.c_size_t(0)
    B.check(L.cf_probe_ws_size(int(kind), C.byref(n)))
    ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device="cuda")
    r = B.cf_probe_result()
    B.check(L.cf_probe(int(kind), ws.data_ptr(), ws.numel(), int(reps), _stream_ptr(stream), C.byref(r)))
    return {"work": r.work, "best_ms": r.best_ms, "rate": r.rate, "sm_mhz": r.sm_mhz, "per_clk_sm": r.per_clk_sm,
            "n_sm": r.n_sm}
