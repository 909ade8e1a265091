// Small kernels: pack edge-weight update from user-order weights, and the
// per-row top-k of the query workload (a9).
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

__global__ void zero_w_kernel(CfAdj* out_adj, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out_adj[e].w = 0.f;
}

// Duplicate user edges add into their one distinct edge.
__global__ void add_w_kernel(CfAdj* out_adj, const int32_t* u2c, const float* w_user, int64_t n_user) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_user; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&out_adj[u2c[e]].w, w_user[e]);
}

__global__ void in_w_kernel(CfAdj* in_adj, const int32_t* in_eid, const CfAdj* out_adj, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    in_adj[k].w = out_adj[in_eid[k]].w;
}

// Order-preserving map of a float to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t float_key(float v) {
  uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

constexpr int kTopkNT = 256;

// One CTA per row: k rounds of a block-wide max over 64-bit keys
// (score key << 32 | ~column), each round below the previous winner, so ties
// go to the smaller column and the result is exact and deterministic.
__global__ void __launch_bounds__(kTopkNT) topk_kernel(const float* scores, int C, int k, float* top, int32_t* idx) {
  __shared__ uint64_t red[kTopkNT / 32];
  const int q = blockIdx.x;
  const float* row = scores + (size_t)q * C;
  uint64_t prev = ~0ull;
  for (int r = 0; r < k; ++r) {
    uint64_t best = 0;
    for (int c = threadIdx.x; c < C; c += kTopkNT) {
      const uint64_t key = ((uint64_t)float_key(row[c]) << 32) | (uint32_t)(~(uint32_t)c);
      if (key < prev && key > best) best = key;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    uint64_t b = 0;
#pragma unroll
    for (int w = 0; w < kTopkNT / 32; ++w) b = red[w] > b ? red[w] : b;
    __syncthreads();
    prev = b;
    if (threadIdx.x == 0) {
      const int c = (int)(~(uint32_t)(b & 0xffffffffu));
      idx[(size_t)q * k + r] = c;
      top[(size_t)q * k + r] = row[c];
    }
  }
}

// The pair list of the winners: pairs[2 (q k + r)] = rows ? rows[q] : q, and
// pairs[2 (q k + r) + 1] = idx[q k + r], for every query q and rank r.
__global__ void topk_pairs_kernel(const int32_t* idx, int Q, int k, const int32_t* rows, int32_t* pairs) {
  const int64_t n = (int64_t)Q * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / k);
    pairs[2 * t] = rows ? rows[q] : q;
    pairs[2 * t + 1] = idx[t];
  }
}

}  // namespace

cudaError_t launch_topk_pairs(const int32_t* idx, int Q, int k, const int32_t* rows, int32_t* pairs, cudaStream_t s) {
  const int64_t n = (int64_t)Q * k;
  const int g = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  if (n > 0) topk_pairs_kernel<<<g, 256, 0, s>>>(idx, Q, k, rows, pairs);
  return cudaGetLastError();
}

cudaError_t launch_set_weights(CfAdj* out_adj, CfAdj* in_adj, const int32_t* in_eid, const int32_t* u2c,
                               int64_t n_user_edges, int64_t n_edges, const float* w_user, cudaStream_t s) {
  const int nt = 256;
  const int g1 = (int)((n_edges + nt - 1) / nt > 0 ? (n_edges + nt - 1) / nt : 1);
  const int g2 = (int)((n_user_edges + nt - 1) / nt > 0 ? (n_user_edges + nt - 1) / nt : 1);
  if (n_edges > 0) zero_w_kernel<<<g1 < 4096 ? g1 : 4096, nt, 0, s>>>(out_adj, n_edges);
  if (n_user_edges > 0) add_w_kernel<<<g2 < 4096 ? g2 : 4096, nt, 0, s>>>(out_adj, u2c, w_user, n_user_edges);
  if (n_edges > 0) in_w_kernel<<<g1 < 4096 ? g1 : 4096, nt, 0, s>>>(in_adj, in_eid, out_adj, n_edges);
  return cudaGetLastError();
}

cudaError_t launch_topk(const float* scores, int Q, int C, int k, float* top, int32_t* idx, cudaStream_t s) {
  topk_kernel<<<Q, kTopkNT, 0, s>>>(scores, C, k, top, idx);
  return cudaGetLastError();
}

}  // namespace cfsim
