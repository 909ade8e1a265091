// a7: the autotuner of the batched forward.  For a pair list it times every
// kernel configuration (tune id: threads per CTA x smallest group level x
// matching policy) on a deterministic sample of the pairs and returns the
// fastest, caching the choice in a text file keyed by the device, the
// attribute width, K, the normalisation and a signature of the sample's cost
// distribution, so that later runs on a similar workload skip the timing.
// Host code only; the timed calls are ordinary cf_similarity calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cfsim.h"
#include "kernels.h"
#include "layout.h"

namespace cfsim {
void set_error_detail(const char* msg);
}

using namespace cfsim;

namespace {

constexpr int kTuneSample = 16384;  // pairs timed per candidate at most
constexpr int kTuneReps = 3;        // timed calls per candidate (after one warm-up)
constexpr float kTuneBudgetMs = 40.f;  // a timed call of the default tune takes about this long at most
constexpr int kTuneMinPairs = 64;

cf_status tfail(cf_status s, const char* fmt, const char* a = "", int b = 0) {
  char buf[512];
  snprintf(buf, sizeof buf, fmt, a, b);
  set_error_detail(buf);
  return s;
}

struct PackHost {
  PackHeader h;
  const int32_t* node_off;
  const int32_t* edge_off;
};

bool read_pack(const void* p, PackHost* out) {
  if (!p) return false;
  std::memcpy(&out->h, p, sizeof(PackHeader));
  if (out->h.magic != kPackMagic || out->h.version != kPackVersion) return false;
  out->node_off = reinterpret_cast<const int32_t*>(static_cast<const char*>(p) + out->h.off_node);
  out->edge_off = reinterpret_cast<const int32_t*>(static_cast<const char*>(p) + out->h.off_edge);
  return true;
}

// The deterministic sample: pair floor(k P / S) for k < S.
std::vector<int32_t> sample_pairs(const int32_t* h_pairs, int32_t P) {
  const int S = std::min<int>(P, kTuneSample);
  std::vector<int32_t> s(2 * (size_t)S);
  for (int k = 0; k < S; ++k) {
    const int64_t p = (int64_t)k * P / S;
    s[2 * k] = h_pairs[2 * p];
    s[2 * k + 1] = h_pairs[2 * p + 1];
  }
  return s;
}

struct TuneLayout {
  size_t sim_ws, pairs, scores, match, total;
};

// Tuner workspace: the sample's similarity workspace, then its pair list,
// scores and matchings.
cf_status tune_layout(const void* h_pack_a, const void* h_pack_b, const std::vector<int32_t>& sp,
                      const cf_params* params, TuneLayout* L) {
  const int S = (int)(sp.size() / 2);
  size_t ws = 0, ws3 = 0;
  cf_status s = cf_similarity_ws_size(h_pack_a, h_pack_b, sp.data(), S, params, &ws);
  if (s) return s;
  cf_params p3 = *params;  // the candidates with deferred matching steps need room for the ranked lists
  p3.flags = 0;
  p3.tune = kFirstDeferTune;
  s = cf_similarity_ws_size(h_pack_a, h_pack_b, sp.data(), S, &p3, &ws3);
  if (s) return s;
  ws = std::max(ws, ws3);
  int64_t m_elems = 0;
  s = cf_out_sizes(h_pack_a, h_pack_b, sp.data(), S, nullptr, &m_elems);
  if (s) return s;
  size_t o = align_up(ws, kAlign);
  L->sim_ws = ws;
  L->pairs = o;
  o = align_up(o + 8 * (size_t)S, kAlign);
  L->scores = o;
  o = align_up(o + 4 * (size_t)S, kAlign);
  L->match = o;
  o = align_up(o + 4 * (size_t)std::max<int64_t>(m_elems, 1), kAlign);
  L->total = o;
  return CF_OK;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

// Cache key: the size of the tune table (ids mean other configurations when
// it changes), device, SM count, attribute stride, K, normalisation, and the
// sample's distribution over cost buckets (two per octave of the
// per-iteration work), each bucket's share rounded to 1/32.
std::string tune_key(const PackHost& A, const PackHost& B, const std::vector<int32_t>& sp, const cf_params* prm) {
  int dev = 0;
  cudaDeviceProp prop{};
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  const int S = (int)(sp.size() / 2);
  std::vector<int> hist(kBuckets, 0);
  for (int k = 0; k < S; ++k) {
    const int a = sp[2 * k], b = sp[2 * k + 1];
    const int64_t na = A.node_off[a + 1] - A.node_off[a], nb = B.node_off[b + 1] - B.node_off[b];
    const int64_t ea = A.edge_off[a + 1] - A.edge_off[a], eb = B.edge_off[b + 1] - B.edge_off[b];
    hist[cost_bucket(na * nb + 2 * ea * eb)]++;
  }
  std::string sig;
  for (int b = 0; b < kBuckets; ++b) {
    const int q = (int)((32.0 * hist[b]) / std::max(S, 1) + 0.5);
    if (q > 0) sig += std::to_string(b) + ":" + std::to_string(q) + ",";
  }
  std::string name = prop.name;
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  char buf[512];
  snprintf(buf, sizeof buf, "abi2c;tunes=%d;dev=%s;sm=%d;Fp=%d;K=%d;norm=%d;sig=%016llx", kNumTunes, name.c_str(),
           prop.multiProcessorCount, A.h.F_pad, prm->K, prm->norm_mode, (unsigned long long)fnv1a(sig));
  return buf;
}

// Cache file: one "key tune ms" line per entry; the last matching line wins.
bool cache_lookup(const char* path, const std::string& key, int* tune, float* ms) {
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[768];
    int t = 0;
    float m = 0.f;
    if (sscanf(line, "%767s %d %f", k, &t, &m) == 3 && key == k && t >= 1 && t <= kNumTunes) {
      *tune = t;
      *ms = m;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int tune, float ms) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %.6f\n", key.c_str(), tune, ms);
  fclose(f);
}

const char* cache_path_or_env(const char* p) {
  if (p && *p) return p;
  const char* e = std::getenv("CF_AUTOTUNE_CACHE");
  return (e && *e) ? e : nullptr;
}

}  // namespace

extern "C" {

int32_t cf_num_tunes(void) { return kNumTunes; }

cf_status cf_tune_describe(int32_t tune, cf_tune_info* out) {
  if (!out) return tfail(CF_ERR_INVALID_ARG, "out is NULL");
  if (tune < 0 || tune > kNumTunes) return tfail(CF_ERR_INVALID_ARG, "tune %s%d out of range", "", tune);
  const Tune t = decode_tune(tune);
  const ClassCfg cc = fwd_class_cfg(t.variant, t.min_cls, t.ranked, t.cluster);
  out->tune = tune;
  out->threads_per_cta = cc.nt;
  out->smallest_group = group_size(t.min_cls, cc);
  out->matching = t.ranked;
  out->cluster = t.cluster;
  set_error_detail("");
  return CF_OK;
}

cf_status cf_autotune_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                              const cf_params* params, size_t* bytes) {
  if (!bytes || !params) return tfail(CF_ERR_INVALID_ARG, "bytes and params are required");
  if (P < 1 || !h_pairs) return tfail(CF_ERR_INVALID_ARG, "need P >= 1 pairs on the host");
  const std::vector<int32_t> sp = sample_pairs(h_pairs, P);
  TuneLayout L{};
  cf_status s = tune_layout(h_pack_a, h_pack_b, sp, params, &L);
  if (s) return s;
  *bytes = L.total;
  set_error_detail("");
  return CF_OK;
}

cf_status cf_autotune(const void* h_pack_a, const void* h_pack_b, const void* d_pack_a, const void* d_pack_b,
                      const int32_t* h_pairs, int32_t P, const cf_params* params, const float* d_omega, void* d_ws,
                      size_t ws_bytes, const char* cache_path, cf_stream_t stream, int32_t* tune, float* best_ms) {
  if (!tune || !params || !d_ws || !d_omega || !d_pack_a || !d_pack_b)
    return tfail(CF_ERR_INVALID_ARG, "tune, params, d_ws, d_omega and the device packs are required");
  if (P < 1 || !h_pairs) return tfail(CF_ERR_INVALID_ARG, "need P >= 1 pairs on the host");
  PackHost A, B;
  if (!read_pack(h_pack_a, &A) || !read_pack(h_pack_b, &B)) return tfail(CF_ERR_INVALID_ARG, "bad host pack");
  const std::vector<int32_t> sp = sample_pairs(h_pairs, P);
  const int S = (int)(sp.size() / 2);
  TuneLayout L{};
  cf_status s = tune_layout(h_pack_a, h_pack_b, sp, params, &L);  // validates packs, pairs and params
  if (s) return s;
  if (ws_bytes < L.total) return tfail(CF_ERR_WORKSPACE, "autotune workspace too small (see cf_autotune_ws_size)");
  const std::string key = tune_key(A, B, sp, params);
  const char* path = cache_path_or_env(cache_path);
  float ms_hit = 0.f;
  int t_hit = 0;
  if (cache_lookup(path, key, &t_hit, &ms_hit)) {
    *tune = t_hit;
    if (best_ms) *best_ms = ms_hit;
    set_error_detail("");
    return CF_OK;
  }

  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(d_ws);
  int32_t* d_pairs = reinterpret_cast<int32_t*>(base + L.pairs);
  float* d_scores = reinterpret_cast<float*>(base + L.scores);
  int32_t* d_match = reinterpret_cast<int32_t*>(base + L.match);
  cudaError_t e = cudaMemcpyAsync(d_pairs, sp.data(), 8 * (size_t)S, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return tfail(CF_ERR_CUDA, "autotune pair upload: %s", cudaGetErrorString(e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return tfail(CF_ERR_CUDA, "autotune events");
  }
  // one timed call of cf_similarity under `tune` on the first n sample pairs
  auto timed = [&](int tune_id, int n, float* ms) -> cf_status {
    cf_params p = *params;
    p.flags = 0;
    p.tune = tune_id;
    cudaEventRecord(e0, st);
    cf_status r = cf_similarity(d_pack_a, d_pack_b, d_pairs, n, &p, d_omega, nullptr, d_scores, d_match, d_ws,
                                L.sim_ws, stream);
    if (r) return r;
    cudaEventRecord(e1, st);
    const cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) return tfail(CF_ERR_CUDA, "autotune run: %s", cudaGetErrorString(ce));
    cudaEventElapsedTime(ms, e0, e1);
    return CF_OK;
  };
  // if one call of the default tune on the sample exceeds the time budget,
  // time the candidates on an evenly strided part of the sample that fits it
  int St = S;
  float ms0 = 0.f;
  s = timed(1, St, &ms0);
  // far over the budget (pairs of hundreds to thousands of blocks): only the
  // thread count and the cluster size matter (such pairs are never
  // shared-memory resident), and the sample is not cut, because a part of it
  // that the device runs in one or two waves favours wide teams (clusters)
  // that lose on the whole batch; one timed call per candidate
  const bool coarse = ms0 > 4.f * kTuneBudgetMs;
  if (s == CF_OK && !coarse && ms0 > kTuneBudgetMs && St > kTuneMinPairs) {
    const int S2 = std::max(kTuneMinPairs, (int)(St * (kTuneBudgetMs / ms0)));
    std::vector<int32_t> sub(2 * (size_t)S2);
    for (int k = 0; k < S2; ++k) {
      const int64_t q = (int64_t)k * St / S2;
      sub[2 * k] = sp[2 * q];
      sub[2 * k + 1] = sp[2 * q + 1];
    }
    if ((e = cudaMemcpyAsync(d_pairs, sub.data(), 8 * (size_t)S2, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      s = tfail(CF_ERR_CUDA, "autotune pair upload: %s", cudaGetErrorString(e));
    St = S2;
  }
  int best_t = 0;
  float best = 1e30f;
  for (int t = 1; t <= kNumTunes && s == CF_OK; ++t) {
    if (coarse) {  // smallest group a warp, ranked lists in groups of at most a quarter CTA
      const Tune d = decode_tune(t);
      if (d.min_cls != kClassWarp || d.ranked != 1) continue;
    }
    float tmin = 1e30f;
    for (int r = 0; r <= (coarse ? 0 : kTuneReps) && s == CF_OK; ++r) {  // call 0 warms up
      float ms = 0.f;
      s = timed(t, St, &ms);
      if (r > 0 || coarse) tmin = std::min(tmin, ms);
    }
    if (s == CF_OK) s = cf_status_check(d_ws, stream);
    if (s == CF_OK && tmin < best) {
      best = tmin;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  cache_store(path, key, best_t, best);
  *tune = best_t;
  if (best_ms) *best_ms = best;
  set_error_detail("");
  return CF_OK;
}

}  // extern "C"
