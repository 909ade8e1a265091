// The C ABI of libcfsim.so (include/cfsim.h): argument validation, the host
// builder of the CSR batch pack (a1), workspace sizing, and the launch
// sequence of every call.  Host code only; kernels live in the other .cu files.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/cfsim.h"
#include "kernels.h"
#include "layout.h"

using namespace cfsim;

namespace {

thread_local std::string g_err;

// An NVTX range ("cfsim/...") around a host-side stretch of a call: pack,
// plan, iterate (the persistent forward with the fused greedy matching),
// match and backward show up on a profiler's timeline with the kernels they
// enqueue.  Without a profiler attached NVTX calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

cf_status fail(cf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

cf_status ok() {
  g_err.clear();
  return CF_OK;
}

cf_status cuda_fail(cudaError_t e, const char* where) {
  return fail(CF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}


// Validate the views and compute the pack layout; when `out` is given, fill it.
cf_status build_pack(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, void* out, size_t out_bytes,
                     size_t* bytes_needed) {
  if (n_cfgs < 1) return fail(CF_ERR_INVALID_ARG, "n_cfgs must be >= 1 (got %d)", n_cfgs);
  if (!cfgs) return fail(CF_ERR_INVALID_ARG, "cfgs is NULL");
  if (F < 1 || F > kMaxF) return fail(CF_ERR_UNSUPPORTED, "F must be in [1, %d] (got %d)", kMaxF, F);
  const int F_pad = (F + 3) / 4 * 4;
  int64_t n_blocks = 0, n_user = 0;
  int max_blocks = 0;
  for (int c = 0; c < n_cfgs; ++c) {
    const cf_cfg_view& v = cfgs[c];
    if (v.n_blocks < 1) return fail(CF_ERR_INVALID_ARG, "cfg %d: n_blocks must be >= 1 (got %d)", c, v.n_blocks);
    if (v.n_blocks > kMaxBlocks)
      return fail(CF_ERR_UNSUPPORTED, "cfg %d: %d blocks exceeds the limit of %d", c, v.n_blocks, kMaxBlocks);
    if (v.n_edges < 0) return fail(CF_ERR_INVALID_ARG, "cfg %d: n_edges < 0", c);
    if (!v.attr) return fail(CF_ERR_INVALID_ARG, "cfg %d: attr is NULL", c);
    if (v.n_edges > 0 && (!v.src || !v.dst || !v.w)) return fail(CF_ERR_INVALID_ARG, "cfg %d: edge array is NULL", c);
    for (int e = 0; e < v.n_edges; ++e) {
      if (v.src[e] < 0 || v.src[e] >= v.n_blocks || v.dst[e] < 0 || v.dst[e] >= v.n_blocks)
        return fail(CF_ERR_INVALID_ARG, "cfg %d edge %d: endpoint out of range (%d -> %d, n_blocks %d)", c, e,
                    v.src[e], v.dst[e], v.n_blocks);
      if (!(std::isfinite(v.w[e]) && v.w[e] >= 0.f))
        return fail(CF_ERR_INVALID_ARG, "cfg %d edge %d: weight must be finite and >= 0", c, e);
    }
    for (int64_t k = 0; k < (int64_t)v.n_blocks * F; ++k)
      if (!(std::isfinite(v.attr[k]) && v.attr[k] >= 0.f))
        return fail(CF_ERR_INVALID_ARG, "cfg %d attribute %lld: must be finite and >= 0", c, (long long)k);
    n_blocks += v.n_blocks;
    n_user += v.n_edges;
    max_blocks = std::max(max_blocks, v.n_blocks);
  }
  if (n_blocks >= INT32_MAX || n_user >= INT32_MAX)
    return fail(CF_ERR_UNSUPPORTED, "pack too large (%lld blocks, %lld edges)", (long long)n_blocks, (long long)n_user);

  // distinct edges per CFG (sorted by (src, dst), duplicates merged)
  std::vector<std::vector<int32_t>> order(n_cfgs);
  std::vector<int32_t> n_distinct(n_cfgs);
  int64_t n_edges = 0;
  for (int c = 0; c < n_cfgs; ++c) {
    const cf_cfg_view& v = cfgs[c];
    std::vector<int32_t>& o = order[c];
    o.resize(v.n_edges);
    std::iota(o.begin(), o.end(), 0);
    std::stable_sort(o.begin(), o.end(), [&](int32_t x, int32_t y) {
      return v.src[x] != v.src[y] ? v.src[x] < v.src[y] : v.dst[x] < v.dst[y];
    });
    int d = 0;
    for (int k = 0; k < v.n_edges; ++k)
      if (k == 0 || v.src[o[k]] != v.src[o[k - 1]] || v.dst[o[k]] != v.dst[o[k - 1]]) ++d;
    n_distinct[c] = d;
    n_edges += d;
  }

  PackHeader h{};
  h.magic = kPackMagic;
  h.version = kPackVersion;
  h.n_cfgs = n_cfgs;
  h.F = F;
  h.F_pad = F_pad;
  h.max_blocks = max_blocks;
  h.n_blocks = n_blocks;
  h.n_edges = n_edges;
  h.n_user_edges = n_user;
  size_t o = align_up(sizeof(PackHeader), kAlign);
  auto take = [&](size_t b) {
    size_t at = o;
    o = align_up(o + b, kAlign);
    return (int64_t)at;
  };
  h.off_node = take(4 * (size_t)(n_cfgs + 1));
  h.off_edge = take(4 * (size_t)(n_cfgs + 1));
  h.off_uedge = take(4 * (size_t)(n_cfgs + 1));
  h.off_out_ptr = take(4 * (size_t)(n_blocks + 1));
  h.off_in_ptr = take(4 * (size_t)(n_blocks + 1));
  h.off_out_adj = take(sizeof(CfAdj) * (size_t)std::max<int64_t>(n_edges, 1));
  h.off_in_adj = take(sizeof(CfAdj) * (size_t)std::max<int64_t>(n_edges, 1));
  h.off_in_eid = take(4 * (size_t)std::max<int64_t>(n_edges, 1));
  h.off_u2c = take(4 * (size_t)std::max<int64_t>(n_user, 1));
  h.off_attr = take(4 * (size_t)n_blocks * F_pad);
  h.off_xdeg = take((size_t)n_cfgs);
  h.total_bytes = (int64_t)o;
  *bytes_needed = o;
  if (!out) return ok();
  if (out_bytes < o) return fail(CF_ERR_WORKSPACE, "pack buffer has %zu bytes, needs %zu", out_bytes, o);

  char* base = static_cast<char*>(out);
  std::memset(base, 0, o);
  int32_t* node_off = reinterpret_cast<int32_t*>(base + h.off_node);
  int32_t* edge_off = reinterpret_cast<int32_t*>(base + h.off_edge);
  int32_t* uedge_off = reinterpret_cast<int32_t*>(base + h.off_uedge);
  int32_t* out_ptr = reinterpret_cast<int32_t*>(base + h.off_out_ptr);
  int32_t* in_ptr = reinterpret_cast<int32_t*>(base + h.off_in_ptr);
  CfAdj* out_adj = reinterpret_cast<CfAdj*>(base + h.off_out_adj);
  CfAdj* in_adj = reinterpret_cast<CfAdj*>(base + h.off_in_adj);
  int32_t* in_eid = reinterpret_cast<int32_t*>(base + h.off_in_eid);
  int32_t* u2c = reinterpret_cast<int32_t*>(base + h.off_u2c);
  float* attr = reinterpret_cast<float*>(base + h.off_attr);
  uint8_t* xdeg = reinterpret_cast<uint8_t*>(base + h.off_xdeg);

  int32_t nb = 0, ne = 0, nu = 0;
  int max_out = 0, max_in = 0;
  for (int c = 0; c < n_cfgs; ++c) {
    const cf_cfg_view& v = cfgs[c];
    node_off[c] = nb;
    edge_off[c] = ne;
    uedge_off[c] = nu;
    const std::vector<int32_t>& ord = order[c];
    // distinct edges in (src, dst) order; u2c for every user edge
    std::vector<int32_t> dsrc, ddst;
    std::vector<float> dw;
    for (int k = 0; k < v.n_edges; ++k) {
      const int e = ord[k];
      if (k == 0 || v.src[e] != v.src[ord[k - 1]] || v.dst[e] != v.dst[ord[k - 1]]) {
        dsrc.push_back(v.src[e]);
        ddst.push_back(v.dst[e]);
        dw.push_back(0.f);
      }
      dw.back() += v.w[e];
      u2c[nu + e] = ne + (int32_t)dsrc.size() - 1;
    }
    const int d = (int)dsrc.size();
    std::vector<int32_t> outdeg(v.n_blocks, 0), indeg(v.n_blocks, 0);
    for (int k = 0; k < d; ++k) {
      outdeg[dsrc[k]]++;
      indeg[ddst[k]]++;
      out_adj[ne + k] = CfAdj{ddst[k], dw[k]};
    }
    int32_t run = ne;
    uint8_t busy = 0;
    for (int i = 0; i < v.n_blocks; ++i) {
      out_ptr[nb + i] = run;
      run += outdeg[i];
      max_out = std::max(max_out, outdeg[i]);
      busy |= (outdeg[i] > 2 || indeg[i] > 2) ? 1 : 0;
    }
    xdeg[c] = busy;
    std::vector<int32_t> by_dst(d);
    std::iota(by_dst.begin(), by_dst.end(), 0);
    std::stable_sort(by_dst.begin(), by_dst.end(), [&](int32_t x, int32_t y) {
      return ddst[x] != ddst[y] ? ddst[x] < ddst[y] : dsrc[x] < dsrc[y];
    });
    for (int k = 0; k < d; ++k) {
      const int e = by_dst[k];
      in_adj[ne + k] = CfAdj{dsrc[e], dw[e]};
      in_eid[ne + k] = ne + e;
    }
    run = ne;
    for (int i = 0; i < v.n_blocks; ++i) {
      in_ptr[nb + i] = run;
      run += indeg[i];
      max_in = std::max(max_in, indeg[i]);
    }
    for (int i = 0; i < v.n_blocks; ++i)
      for (int f = 0; f < F; ++f) attr[(size_t)(nb + i) * F_pad + f] = v.attr[(size_t)i * F + f];
    nb += v.n_blocks;
    ne += d;
    nu += v.n_edges;
  }
  node_off[n_cfgs] = nb;
  edge_off[n_cfgs] = ne;
  uedge_off[n_cfgs] = nu;
  out_ptr[nb] = ne;
  in_ptr[nb] = ne;
  h.max_out_deg = max_out;
  h.max_in_deg = max_in;
  std::memcpy(base, &h, sizeof h);
  return ok();
}

cf_status read_header(const void* h_pack, PackHeader* h, const char* what) {
  if (!h_pack) return fail(CF_ERR_INVALID_ARG, "%s is NULL", what);
  std::memcpy(h, h_pack, sizeof *h);
  if (h->magic != kPackMagic || h->version != kPackVersion)
    return fail(CF_ERR_INVALID_ARG, "%s is not a cfsim pack (bad magic/version)", what);
  return CF_OK;
}

cf_status check_params(const cf_params* p) {
  if (!p) return fail(CF_ERR_INVALID_ARG, "params is NULL");
  if (!(p->alpha >= 0.f && p->alpha < 1.f)) return fail(CF_ERR_INVALID_ARG, "alpha must be in [0, 1) (got %g)", p->alpha);
  if (p->K < 0 || p->K > 1000000) return fail(CF_ERR_INVALID_ARG, "K must be in [0, 1e6] (got %d)", p->K);
  if (p->norm_mode != CF_NORM_FROB && p->norm_mode != CF_NORM_NONE)
    return fail(CF_ERR_INVALID_ARG, "unknown norm_mode %d", p->norm_mode);
  if (p->match_mode != CF_MATCH_GREEDY && p->match_mode != CF_MATCH_OPTIMAL)
    return fail(CF_ERR_INVALID_ARG, "unknown match_mode %d", p->match_mode);
  const uint32_t known = CF_FLAG_PER_PAIR_LAUNCH | CF_FLAG_PLAN_ONLY | CF_FLAG_REUSE_PLAN | CF_FLAG_OPT_UNSTAGED |
                         CF_FLAG_PER_PAIR_STREAMS;
  if (p->flags & ~known) return fail(CF_ERR_INVALID_ARG, "unknown flags 0x%x", p->flags);
  if ((p->flags & CF_FLAG_PLAN_ONLY) && (p->flags & CF_FLAG_REUSE_PLAN))
    return fail(CF_ERR_INVALID_ARG, "CF_FLAG_PLAN_ONLY and CF_FLAG_REUSE_PLAN exclude each other");
  if (p->tune < 0 || p->tune > kNumTunes) return fail(CF_ERR_INVALID_ARG, "tune must be in [0, %d] (got %d)", kNumTunes, p->tune);
  return CF_OK;
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Scan the host pair list: validate and size the scratch slots of
// global-class pairs (the class set is the same for the batched and the
// per-pair forms).
cf_status scan_pairs(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                     int64_t* x_elems, int64_t* m_elems, size_t* slot_need, int64_t* n_global) {
  PackHeader ha, hb;
  cf_status s = read_header(h_pack_a, &ha, "h_pack_a");
  if (s) return s;
  s = read_header(h_pack_b, &hb, "h_pack_b");
  if (s) return s;
  if (ha.F != hb.F) return fail(CF_ERR_INVALID_ARG, "packs have different F (%d vs %d)", ha.F, hb.F);
  if (P < 0) return fail(CF_ERR_INVALID_ARG, "P < 0");
  if (P > 0 && !h_pairs) return fail(CF_ERR_INVALID_ARG, "h_pairs is NULL");
  const int32_t* noa = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_a) + ha.off_node);
  const int32_t* nob = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_b) + hb.off_node);
  const int32_t* eoa = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_a) + ha.off_edge);
  const int32_t* eob = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_b) + hb.off_edge);
  const uint8_t* xda = reinterpret_cast<const uint8_t*>(static_cast<const char*>(h_pack_a) + ha.off_xdeg);
  const uint8_t* xdb = reinterpret_cast<const uint8_t*>(static_cast<const char*>(h_pack_b) + hb.off_xdeg);
  int64_t xs = 0, ms = 0, ng = 0;
  size_t need = 0;
  // pairs that fit no single CTA: the global class, or the cluster class under a tune with clusters
  const ClassCfg cc = fwd_class_cfg(0, kClassWarp, 0, 0);
  for (int p = 0; p < P; ++p) {
    const int a = h_pairs[2 * p], b = h_pairs[2 * p + 1];
    if (a < 0 || a >= ha.n_cfgs || b < 0 || b >= hb.n_cfgs)
      return fail(CF_ERR_INVALID_ARG, "pair %d = (%d, %d) out of range (%d x %d CFGs)", p, a, b, ha.n_cfgs, hb.n_cfgs);
    const int na = noa[a + 1] - noa[a], nb = nob[b + 1] - nob[b];
    xs += (int64_t)na * nb;
    ms += na;
    if (classify(na, nb, eoa[a + 1] - eoa[a], eob[b + 1] - eob[b], cc, xda[a], xdb[b]).cls == kClassGlobal) {
      need = std::max(need, global_slot_bytes(na, nb));
      ++ng;
    }
  }
  if (x_elems) *x_elems = xs;
  if (m_elems) *m_elems = ms;
  if (slot_need) *slot_need = need;
  if (n_global) *n_global = ng;
  return CF_OK;
}

}  // namespace

namespace cfsim {
// Kernel configuration of a tune id (cf_params.tune): 0 is the built-in
// default (same as id 1); ids 1..kNumTunes enumerate variant x smallest group
// level x matching policy x cluster size of the cluster tier.
Tune decode_tune(int32_t id) {
  static const int kClusters[4] = {0, 2, 4, 8};
  const int idx = id >= 1 && id <= kNumTunes ? id - 1 : 0;
  Tune t;
  if (idx >= kFirstDeferTune - 1) {  // matching policy 3: variant x smallest group x cluster size
    const int j = idx - (kFirstDeferTune - 1);
    t.variant = j % 3;
    t.min_cls = kClassWarp - (j / 3) % 5;
    t.ranked = 3;
    t.cluster = kClusters[j / 15];
    return t;
  }
  t.variant = idx % 3;
  t.min_cls = kClassWarp - (idx / 3) % 5;
  t.ranked = (idx / 15) % 3;
  t.cluster = kClusters[idx / 45];
  return t;
}
}  // namespace cfsim

namespace {

// Kernel configuration of the adjoint: tune 0 is its default (512 threads,
// clusters of kBwdDefaultCluster CTAs for the pairs that fit no single CTA:
// the fastest measured on the 256-pair gradient workload); another tune id
// gives its thread count (1024 runs as 768, which the adjoint is built for)
// and cluster size.
constexpr int kBwdDefaultCluster = 8;
void bwd_config(const cf_params* p, int* variant, int* cluster) {
  if (!p || p->tune == 0) {
    *variant = 1;
    *cluster = kBwdDefaultCluster;
    return;
  }
  const Tune t = decode_tune(p->tune);
  *variant = t.variant == 1 ? 1 : 2;
  *cluster = t.cluster;
}

CallArgs base_args(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                   const cf_params* params, const float* d_omega, void* d_ws, size_t ws_bytes) {
  CallArgs a{};
  a.pack_a = d_pack_a;
  a.pack_b = d_pack_b;
  a.pairs = d_pairs;
  a.P = P;
  const Tune tn = decode_tune(params ? params->tune : 0);
  a.min_cls = tn.min_cls;
  a.ranked = tn.ranked;
  a.cluster = 0;
  if (params) {
    a.alpha = params->alpha;
    a.K = params->K;
    a.norm_mode = params->norm_mode;
    a.opt_unstaged = (params->flags & CF_FLAG_OPT_UNSTAGED) ? 1 : 0;
    a.pp_streams = (params->flags & CF_FLAG_PER_PAIR_STREAMS) ? kPerPairStreams : 0;
  }
  a.omega = d_omega;
  a.ws = static_cast<unsigned char*>(d_ws);
  a.ws_bytes = ws_bytes;
  return a;
}

cf_status check_device_call(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                            void* d_ws, size_t ws_bytes) {
  if (P < 0) return fail(CF_ERR_INVALID_ARG, "P < 0");
  if (!d_pack_a || !d_pack_b) return fail(CF_ERR_INVALID_ARG, "device pack is NULL");
  if (P > 0 && !d_pairs) return fail(CF_ERR_INVALID_ARG, "d_pairs is NULL");
  if (!d_ws) return fail(CF_ERR_INVALID_ARG, "d_ws is NULL");
  const size_t fixed = ws_layout(P).fixed_bytes;
  if (ws_bytes < fixed) return fail(CF_ERR_WORKSPACE, "workspace has %zu bytes, needs at least %zu", ws_bytes, fixed);
  return CF_OK;
}

}  // namespace

namespace cfsim {
// Set the calling thread's error detail from another translation unit.
void set_error_detail(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace cfsim

extern "C" {

const char* cf_status_string(cf_status s) {
  switch (s) {
    case CF_OK: return "ok";
    case CF_ERR_INVALID_ARG: return "invalid argument";
    case CF_ERR_WORKSPACE: return "workspace or buffer too small";
    case CF_ERR_UNSUPPORTED: return "unsupported input";
    case CF_ERR_CUDA: return "CUDA error";
    case CF_ERR_TIMEOUT: return "device wait timed out";
    case CF_ERR_NUMERIC: return "non-finite or negative value on the device";
  }
  return "unknown status";
}

const char* cf_last_error_detail(void) { return g_err.c_str(); }

int32_t cf_abi_version(void) { return 2; }

cf_status cf_pack_size(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, size_t* bytes) {
  if (!bytes) return fail(CF_ERR_INVALID_ARG, "bytes is NULL");
  return build_pack(cfgs, n_cfgs, F, nullptr, 0, bytes);
}

cf_status cf_pack_host(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, void* h_pack, size_t bytes) {
  size_t need = 0;
  if (!h_pack) return fail(CF_ERR_INVALID_ARG, "h_pack is NULL");
  return build_pack(cfgs, n_cfgs, F, h_pack, bytes, &need);
}

cf_status cf_pack_info_get(const void* h_pack, cf_pack_info* info) {
  PackHeader h;
  cf_status s = read_header(h_pack, &h, "h_pack");
  if (s) return s;
  if (!info) return fail(CF_ERR_INVALID_ARG, "info is NULL");
  info->n_cfgs = h.n_cfgs;
  info->F = h.F;
  info->F_pad = h.F_pad;
  info->max_blocks = h.max_blocks;
  info->n_blocks = h.n_blocks;
  info->n_edges = h.n_edges;
  info->n_user_edges = h.n_user_edges;
  info->bytes = h.total_bytes;
  return ok();
}

cf_status cf_pack_cfgs(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, void* d_pack, size_t bytes,
                       cf_stream_t stream) {
  NvtxRange nv("cfsim/pack");
  size_t need = 0;
  cf_status s = build_pack(cfgs, n_cfgs, F, nullptr, 0, &need);
  if (s) return s;
  if (!d_pack) return fail(CF_ERR_INVALID_ARG, "d_pack is NULL");
  if (bytes < need) return fail(CF_ERR_WORKSPACE, "d_pack has %zu bytes, needs %zu", bytes, need);
  std::vector<unsigned char> host(need);
  s = build_pack(cfgs, n_cfgs, F, host.data(), need, &need);
  if (s) return s;
  cudaError_t e = cudaMemcpyAsync(d_pack, host.data(), need, cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cf_pack_cfgs copy");
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cf_pack_cfgs sync");
  return ok();
}

cf_status cf_pack_set_weights(void* d_pack, const void* h_pack, const float* d_w_user, cf_stream_t stream) {
  PackHeader h;
  cf_status s = read_header(h_pack, &h, "h_pack");
  if (s) return s;
  if (!d_pack) return fail(CF_ERR_INVALID_ARG, "d_pack is NULL");
  if (h.n_user_edges > 0 && !d_w_user) return fail(CF_ERR_INVALID_ARG, "d_w_user is NULL");
  char* b = static_cast<char*>(d_pack);
  cudaError_t e = launch_set_weights(reinterpret_cast<CfAdj*>(b + h.off_out_adj), reinterpret_cast<CfAdj*>(b + h.off_in_adj),
                                     reinterpret_cast<const int32_t*>(b + h.off_in_eid),
                                     reinterpret_cast<const int32_t*>(b + h.off_u2c), h.n_user_edges, h.n_edges,
                                     d_w_user, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cf_pack_set_weights");
  return ok();
}

cf_status cf_out_sizes(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                       int64_t* x_elems, int64_t* match_elems) {
  cf_status s = scan_pairs(h_pack_a, h_pack_b, h_pairs, P, x_elems, match_elems, nullptr, nullptr);
  return s ? s : ok();
}

cf_status cf_similarity_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                                const cf_params* params, size_t* bytes) {
  if (!bytes) return fail(CF_ERR_INVALID_ARG, "bytes is NULL");
  if (params) {
    cf_status s = check_params(params);
    if (s) return s;
  }
  size_t need = 0;
  int64_t ng = 0, xs = 0;
  cf_status s = scan_pairs(h_pack_a, h_pack_b, h_pairs, P, &xs, nullptr, &need, &ng);
  if (s) return s;
  // scratch slots for global-class pairs: one per concurrently working CTA
  // (the plain form spread over streams: one per stream)
  int sms = device_sm_count();
  int64_t slots = std::min<int64_t>(ng, 2 * (sms > 0 ? sms : 152));
  if (params && (params->flags & CF_FLAG_PER_PAIR_STREAMS) && ng > 0) slots = std::max<int64_t>(slots, kPerPairStreams);
  *bytes = ws_layout(P).fixed_bytes + (size_t)slots * need;
  // matching policy 3: room for every pair's ranked lists (deferred steps)
  if (params && decode_tune(params->tune).ranked == 3 && !(params->flags & CF_FLAG_PER_PAIR_LAUNCH))
    *bytes += defer_bytes(P, xs);
  return ok();
}

cf_status cf_similarity(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                        const cf_params* params, const float* d_omega, float* d_X, float* d_scores,
                        int32_t* d_match, void* d_ws, size_t ws_bytes, cf_stream_t stream) {
  cf_status s = check_params(params);
  if (s) return s;
  s = check_device_call(d_pack_a, d_pack_b, d_pairs, P, d_ws, ws_bytes);
  if (s) return s;
  if (!d_omega) return fail(CF_ERR_INVALID_ARG, "d_omega is NULL");
  const bool optimal = params->match_mode == CF_MATCH_OPTIMAL && (d_scores || d_match);
  if (optimal && !d_X)
    return fail(CF_ERR_INVALID_ARG, "CF_MATCH_OPTIMAL runs on the matrices: d_X is required with d_scores / d_match");
  if (P == 0) return ok();
  CallArgs a = base_args(d_pack_a, d_pack_b, d_pairs, P, params, d_omega, d_ws, ws_bytes);
  a.X = d_X;
  a.scores = optimal ? nullptr : d_scores;
  a.match = optimal ? nullptr : d_match;
  const Tune tn = decode_tune(params->tune);
  // the cluster tier only in the batched form, and only where such clusters can be resident
  if (!(params->flags & CF_FLAG_PER_PAIR_LAUNCH) && tn.cluster >= 2) a.cluster = cluster_supported(tn.variant, tn.cluster);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (params->flags & CF_FLAG_REUSE_PLAN) {
    // only the queue cursors restart; the plan and the status word stay
    e = cudaMemsetAsync(static_cast<char*>(d_ws) + offsetof(WsHeader, q_next), 0, sizeof(uint32_t) * kNumClasses, st);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    e = cudaMemsetAsync(static_cast<char*>(d_ws) + offsetof(WsHeader, n_def), 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
  } else {
    NvtxRange nv("cfsim/plan");
    e = cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st);
    if (e != cudaSuccess) return cuda_fail(e, "workspace reset");
    e = launch_plan(a, fwd_class_cfg(tn.variant, a.min_cls, a.ranked, a.cluster), st);
    if (e != cudaSuccess) return cuda_fail(e, "plan launch");
  }
  if (!(params->flags & CF_FLAG_PLAN_ONLY)) {
    NvtxRange nv("cfsim/iterate");
    e = launch_forward(a, tn.variant, (params->flags & CF_FLAG_PER_PAIR_LAUNCH) != 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    if (tn.ranked == 3 && (a.scores || a.match)) {  // the deferred steps (a no-op if the plan found no room)
      e = launch_match_deferred(a, st);
      if (e != cudaSuccess) return cuda_fail(e, "deferred matching launch");
    }
    if (optimal) {
      if (params->flags & CF_FLAG_REUSE_PLAN) {
        e = cudaMemsetAsync(static_cast<char*>(d_ws) + offsetof(WsHeader, q_opt), 0, sizeof(uint64_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "queue reset");
      }
      a.X_in = d_X;
      a.scores = d_scores;
      a.match = d_match;
      NvtxRange nm("cfsim/match");
      e = launch_match_optimal(a, st);
      if (e != cudaSuccess) return cuda_fail(e, "optimal matching launch");
    }
  }
  return ok();
}

cf_status cf_match(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                   const cf_params* params, const float* d_omega, const float* d_X_in, int32_t* d_match,
                   float* d_scores, void* d_ws, size_t ws_bytes, cf_stream_t stream) {
  if (!d_X_in) return cf_similarity(d_pack_a, d_pack_b, d_pairs, P, params, d_omega, nullptr, d_scores, d_match,
                                    d_ws, ws_bytes, stream);
  NvtxRange nv("cfsim/match");
  cf_status s = check_device_call(d_pack_a, d_pack_b, d_pairs, P, d_ws, ws_bytes);
  if (s) return s;
  if (params && params->match_mode != CF_MATCH_GREEDY && params->match_mode != CF_MATCH_OPTIMAL)
    return fail(CF_ERR_INVALID_ARG, "unknown match_mode %d", params->match_mode);
  if (P == 0) return ok();
  CallArgs a = base_args(d_pack_a, d_pack_b, d_pairs, P, nullptr, nullptr, d_ws, ws_bytes);
  a.opt_unstaged = params && (params->flags & CF_FLAG_OPT_UNSTAGED) ? 1 : 0;
  a.X_in = d_X_in;
  a.scores = d_scores;
  a.match = d_match;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "workspace reset");
  e = launch_plan(a, fwd_class_cfg(0, a.min_cls, a.ranked, 0), st);
  if (e != cudaSuccess) return cuda_fail(e, "plan launch");
  if (params && params->match_mode == CF_MATCH_OPTIMAL)
    e = launch_match_optimal(a, st);
  else
    e = launch_match_only(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "match launch");
  return ok();
}

cf_status cf_similarity_backward_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs,
                                         int32_t P, const cf_params* params, size_t* bytes) {
  if (!bytes) return fail(CF_ERR_INVALID_ARG, "bytes is NULL");
  cf_status s = check_params(params);
  if (s) return s;
  PackHeader ha, hb;
  s = read_header(h_pack_a, &ha, "h_pack_a");
  if (s) return s;
  s = read_header(h_pack_b, &hb, "h_pack_b");
  if (s) return s;
  s = scan_pairs(h_pack_a, h_pack_b, h_pairs, P, nullptr, nullptr, nullptr, nullptr);
  if (s) return s;
  int variant = 0, cluster = 0;
  bwd_config(params, &variant, &cluster);
  const BwdShape sh = bwd_shape(variant, cluster, params->K);
  if (sh.n_cta <= 0) return fail(CF_ERR_CUDA, "cf_similarity_backward_ws_size: no usable CUDA device");
  const int32_t* noa = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_a) + ha.off_node);
  const int32_t* nob = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_b) + hb.off_node);
  const int32_t* eoa = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_a) + ha.off_edge);
  const int32_t* eob = reinterpret_cast<const int32_t*>(static_cast<const char*>(h_pack_b) + hb.off_edge);
  const uint8_t* xda = reinterpret_cast<const uint8_t*>(static_cast<const char*>(h_pack_a) + ha.off_xdeg);
  const uint8_t* xdb = reinterpret_cast<const uint8_t*>(static_cast<const char*>(h_pack_b) + hb.off_xdeg);
  // the classification of the device-side plan: pairs that fit no single CTA
  // need a team slot (the largest such pair sizes them)
  size_t need = 0;
  int64_t n_big = 0;
  for (int p = 0; p < P; ++p) {
    const int a = h_pairs[2 * p], b = h_pairs[2 * p + 1];
    const int na = noa[a + 1] - noa[a], nb = nob[b + 1] - nob[b];
    const int ea = eoa[a + 1] - eoa[a], eb = eob[b + 1] - eob[b];
    const Shape sp = classify(na, nb, ea, eb, sh.cc, xda[a], xdb[b]);
    if (sp.cls == kClassGlobal) {
      need = std::max(need, bwd_slot_bytes(na, nb, ea, eb, params->K, ha.F_pad));
      ++n_big;
    } else if (sp.cls == kClassCluster) {
      need = std::max(need, bwd_res_slot_bytes(sp.n_row, sp.ld, params->K));
      ++n_big;
    }
  }
  const int64_t slots = std::min<int64_t>(n_big, sh.n_teams);
  // sized as if the two sides were different packs (covers both cases)
  *bytes = bwd_layout(P, ha.n_edges, hb.n_edges, false).slots + (size_t)sh.n_cta * sh.area_bytes + (size_t)slots * need;
  return ok();
}

cf_status cf_similarity_backward(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                                 const cf_params* params, const float* d_omega, const int32_t* d_match,
                                 const float* d_grad_scores, float* d_grad_w_a, float* d_grad_w_b,
                                 float* d_grad_omega, void* d_ws, size_t ws_bytes, cf_stream_t stream) {
  cf_status s = check_params(params);
  if (s) return s;
  if (params->flags & (CF_FLAG_PER_PAIR_LAUNCH | CF_FLAG_PLAN_ONLY | CF_FLAG_REUSE_PLAN))
    return fail(CF_ERR_INVALID_ARG, "cf_similarity_backward takes no launch flags");
  s = check_device_call(d_pack_a, d_pack_b, d_pairs, P, d_ws, ws_bytes);
  if (s) return s;
  if (!d_omega || !d_match || !d_grad_scores) return fail(CF_ERR_INVALID_ARG, "d_omega, d_match and d_grad_scores are required");
  if (d_pack_a == d_pack_b && d_grad_w_b && d_grad_w_b != d_grad_w_a)
    return fail(CF_ERR_INVALID_ARG, "with one pack on both sides, d_grad_w_b must be NULL or equal d_grad_w_a");
  if (P == 0) return ok();
  NvtxRange nv("cfsim/backward");
  int variant = 0, cluster = 0;
  bwd_config(params, &variant, &cluster);
  const BwdShape sh = bwd_shape(variant, cluster, params->K);
  if (sh.n_cta <= 0) return fail(CF_ERR_CUDA, "cf_similarity_backward: no usable CUDA device");
  CallArgs a = base_args(d_pack_a, d_pack_b, d_pairs, P, params, d_omega, d_ws, ws_bytes);
  a.match_in = d_match;
  a.grad_scores = d_grad_scores;
  a.grad_w_a = d_grad_w_a;
  a.grad_w_b = d_pack_a == d_pack_b ? nullptr : d_grad_w_b;
  a.grad_omega = d_grad_omega;
  a.cluster = sh.cluster;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "workspace reset");
  e = launch_plan(a, sh.cc, st);
  if (e != cudaSuccess) return cuda_fail(e, "plan launch");
  e = launch_backward(a, variant, st);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return ok();
}

cf_status cf_topk(const float* d_scores, int32_t Q, int32_t C, int32_t k, float* d_top, int32_t* d_idx,
                  cf_stream_t stream) {
  if (Q < 0 || C < 1 || k < 1 || k > C || k > 1024)
    return fail(CF_ERR_INVALID_ARG, "need Q >= 0, 1 <= k <= min(C, 1024) (Q=%d C=%d k=%d)", Q, C, k);
  if (Q == 0) return ok();
  if (!d_scores || !d_top || !d_idx) return fail(CF_ERR_INVALID_ARG, "NULL buffer");
  cudaError_t e = launch_topk(d_scores, Q, C, k, d_top, d_idx, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "topk launch");
  return ok();
}

cf_status cf_topk_pairs(const int32_t* d_idx, int32_t Q, int32_t k, const int32_t* d_rows, int32_t* d_pairs,
                        cf_stream_t stream) {
  if (Q < 0 || k < 1) return fail(CF_ERR_INVALID_ARG, "need Q >= 0 and k >= 1 (Q=%d k=%d)", Q, k);
  if (Q == 0) return ok();
  if (!d_idx || !d_pairs) return fail(CF_ERR_INVALID_ARG, "NULL buffer");
  cudaError_t e = launch_topk_pairs(d_idx, Q, k, d_rows, d_pairs, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "topk pairs launch");
  return ok();
}

cf_status cf_similarity_ws_size_any(const void* h_pack_a, const void* h_pack_b, int32_t P, const cf_params* params,
                                    size_t* bytes) {
  if (!bytes) return fail(CF_ERR_INVALID_ARG, "bytes is NULL");
  if (P < 0) return fail(CF_ERR_INVALID_ARG, "P < 0");
  if (params) {
    cf_status s = check_params(params);
    if (s) return s;
  }
  PackHeader ha, hb;
  cf_status s = read_header(h_pack_a, &ha, "h_pack_a");
  if (s) return s;
  s = read_header(h_pack_b, &hb, "h_pack_b");
  if (s) return s;
  if (ha.F != hb.F) return fail(CF_ERR_INVALID_ARG, "packs have different F (%d vs %d)", ha.F, hb.F);
  // every pair may be as large as the two largest CFGs, and every one may
  // need a scratch slot (at most one per concurrently working CTA)
  const int sms = device_sm_count();
  const int64_t slots = std::min<int64_t>(P, 2 * (sms > 0 ? sms : 152));
  *bytes = ws_layout(P).fixed_bytes + (size_t)slots * global_slot_bytes(ha.max_blocks, hb.max_blocks);
  if (params && decode_tune(params->tune).ranked == 3 && !(params->flags & CF_FLAG_PER_PAIR_LAUNCH))
    *bytes += defer_bytes(P, (int64_t)P * ha.max_blocks * hb.max_blocks);
  return ok();
}

cf_status cf_status_check(const void* d_ws, cf_stream_t stream) {
  if (!d_ws) return fail(CF_ERR_INVALID_ARG, "d_ws is NULL");
  int32_t st[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(st, d_ws, sizeof st, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "status sync");
  if (st[0] != 0)
    return fail((cf_status)st[0], "device reported: %s (detail %d)", cf_status_string((cf_status)st[0]), st[1]);
  return ok();
}

}  // extern "C"
