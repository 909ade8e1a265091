// Device helpers shared by the kernels: resolved pack views, status word,
// warp/CTA reductions and the two thread-group shapes a pair runs on.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "layout.h"

namespace cfsim {

// Pointers into a pack, resolved from its header on the device.
struct PackView {
  const int32_t* node_off;
  const int32_t* edge_off;
  const int32_t* uedge_off;
  const int32_t* out_ptr;
  const int32_t* in_ptr;
  const CfAdj* out_adj;
  const CfAdj* in_adj;
  const int32_t* in_eid;
  const int32_t* u2c;
  const float* attr;
  int n_cfgs, F, F_pad;
};

__device__ __forceinline__ PackView load_pack(const void* base) {
  const PackHeader* h = reinterpret_cast<const PackHeader*>(base);
  const char* b = reinterpret_cast<const char*>(base);
  PackView v;
  v.node_off = reinterpret_cast<const int32_t*>(b + h->off_node);
  v.edge_off = reinterpret_cast<const int32_t*>(b + h->off_edge);
  v.uedge_off = reinterpret_cast<const int32_t*>(b + h->off_uedge);
  v.out_ptr = reinterpret_cast<const int32_t*>(b + h->off_out_ptr);
  v.in_ptr = reinterpret_cast<const int32_t*>(b + h->off_in_ptr);
  v.out_adj = reinterpret_cast<const CfAdj*>(b + h->off_out_adj);
  v.in_adj = reinterpret_cast<const CfAdj*>(b + h->off_in_adj);
  v.in_eid = reinterpret_cast<const int32_t*>(b + h->off_in_eid);
  v.u2c = reinterpret_cast<const int32_t*>(b + h->off_u2c);
  v.attr = reinterpret_cast<const float*>(b + h->off_attr);
  v.n_cfgs = h->n_cfgs;
  v.F = h->F;
  v.F_pad = h->F_pad;
  return v;
}

// Read-only (non-coherent path) load of an adjacency entry.
__device__ __forceinline__ CfAdj ldg_adj(const CfAdj* p) {
  int2 v = __ldg(reinterpret_cast<const int2*>(p));
  CfAdj a;
  a.nbr = v.x;
  a.w = __int_as_float(v.y);
  return a;
}

// Record the first device-side error of a call.
__device__ __forceinline__ void set_status(WsHeader* h, int code, int info) {
  if (atomicCAS(&h->status, 0, code) == 0) h->status_info = info;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;  // every lane holds the same bits (each butterfly step adds a symmetric pair)
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp argmax under the order (value descending, index ascending).
__device__ __forceinline__ void warp_argmax(float& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (v2 > v || (v2 == v && i2 < i)) {
      v = v2;
      i = i2;
    }
  }
}

// A warp working on one pair on its own.
struct WarpGrp {
  int lane;
  __device__ __forceinline__ int rank() const { return lane; }
  static constexpr int size() { return 32; }
  __device__ __forceinline__ int warp() const { return 0; }
  static constexpr int nwarps() { return 1; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  // Sum over the group; every thread gets the same value.  `red`/`par` unused.
  __device__ __forceinline__ float sum(float v, float*, int) const {
    v = warp_sum(v);
    __syncwarp();
    return v;
  }
  __device__ __forceinline__ int sum_i(int v, int*, int) const {
    v = warp_sum_i(v);
    __syncwarp();
    return v;
  }
};

// A whole CTA working on one pair.  sum() contains the group's one barrier;
// `red` holds two parities of per-warp partials so that consecutive sums
// need no second barrier.
template <int NT>
struct CtaGrp {
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  static constexpr int size() { return NT; }
  __device__ __forceinline__ int warp() const { return threadIdx.x >> 5; }
  static constexpr int nwarps() { return NT / 32; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ float sum(float v, float* red, int par) const {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[par * 32 + (threadIdx.x >> 5)] = v;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += red[par * 32 + w];
    return t;
  }
  __device__ __forceinline__ int sum_i(int v, int* red, int par) const {
    v = warp_sum_i(v);
    if ((threadIdx.x & 31) == 0) red[par * 32 + (threadIdx.x >> 5)] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += red[par * 32 + w];
    return t;
  }
};

}  // namespace cfsim
