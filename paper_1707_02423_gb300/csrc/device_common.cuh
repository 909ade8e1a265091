// Device helpers shared by the kernels: resolved pack views, status word,
// warp reductions, named barriers and the weighted attribute products.
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
  const uint8_t* xdeg;
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
  v.xdeg = reinterpret_cast<const uint8_t*>(b + h->off_xdeg);
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

// Debug builds (compiled with -DCF_DEBUG_BOUNDS): checks of each pair's
// shared-memory layout against its region, of scratch slots against the
// workspace, and of staged neighbour indices against the CFG sizes.  A failed
// check records CF_ERR_INVALID_ARG with the check's site code (>= 1000) in
// the status word, and the caller skips the access.  In a normal build every
// check is the constant true and compiles away.
#ifdef CF_DEBUG_BOUNDS
__device__ __forceinline__ bool bounds_ok(WsHeader* h, bool ok, int site) {
  if (!ok && h) set_status(h, 1 /* CF_ERR_INVALID_ARG */, site);
  return ok;
}
#else
__device__ __forceinline__ bool bounds_ok(WsHeader*, bool, int) { return true; }
#endif
enum BoundsSite : int {
  kSiteFwdRegion = 1001,  // a resident pair's layout exceeds its group's region
  kSiteFwdRowNbr = 1002,  // a staged row neighbour outside the row graph
  kSiteFwdColNbr = 1003,  // a staged column neighbour outside the column graph
  kSiteFwdSlot = 1004,    // a global-class scratch slot past the workspace end
  kSiteBwdRegion = 1011,  // an adjoint pair's layout exceeds its region
  kSiteBwdSlot = 1012,    // an adjoint pair's slot exceeds its group's slot
  kSiteBwdRowNbr = 1013,
  kSiteBwdColNbr = 1014
};

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

// Warp argmin under the order (value ascending, index ascending).
__device__ __forceinline__ void warp_argmin(float& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (v2 < v || (v2 == v && i2 < i)) {
      v = v2;
      i = i2;
    }
  }
}

__device__ __forceinline__ void bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Thread-block cluster helpers (PTX): rank and size of the cluster, cluster
// index, the shared::cluster address of a shared-memory location in another
// CTA of the cluster, a full cluster barrier and distributed-shared-memory loads.
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// All threads of all CTAs of the cluster; release / acquire at cluster scope.
// The CTAs of a cluster are co-scheduled, so every arrival happens.
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float cl_ld_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Weighted attribute norm sqrt(sum_f w_f a_f^2) and weighted dot product
// sum_f w_f a_f b_f over the zero-padded F_pad columns, four at a time.
__device__ __forceinline__ float attr_norm(const float* a, const float* om, int Fp) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* o4 = reinterpret_cast<const float4*>(om);
  float acc = 0.f;
  for (int q = 0; q < (Fp >> 2); ++q) {
    const float4 v = __ldg(a4 + q), w = o4[q];
    acc = fmaf(w.x * v.x, v.x, acc);
    acc = fmaf(w.y * v.y, v.y, acc);
    acc = fmaf(w.z * v.z, v.z, acc);
    acc = fmaf(w.w * v.w, v.w, acc);
  }
  return sqrtf(acc);
}

__device__ __forceinline__ float attr_dot(const float* a, const float* b, const float* om, int Fp) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  const float4* o4 = reinterpret_cast<const float4*>(om);
  float acc = 0.f;
  for (int q = 0; q < (Fp >> 2); ++q) {
    const float4 u = __ldg(a4 + q), v = __ldg(b4 + q), w = o4[q];
    acc = fmaf(w.x * u.x, v.x, acc);
    acc = fmaf(w.y * u.y, v.y, acc);
    acc = fmaf(w.z * u.z, v.z, acc);
    acc = fmaf(w.w * u.w, v.w, acc);
  }
  return acc;
}

}  // namespace cfsim
