// Device pieces shared by the forward and the adjoint kernels for pairs whose
// iterates are resident in shared memory (one CTA's group, or the CTAs of a
// thread-block cluster): thread groups with named barriers, the column lists
// each thread keeps in registers, the straight-line neighbour-pair gather and
// its further-neighbour terms, unit attribute vectors, and cluster-wide sums.
//
// The gathered quantity at entry (i, j) is
//   sum_{i->u} sum_{j->v} w_iu w_jv Y[u,v] + sum_{u->i} sum_{v->j} w_ui w_vj Y[u,v],
// the operator M of the iteration (Table 1 "Iso" row read as IsoRank on the
// two weighted CFGs), which is its own adjoint.
#pragma once

#include "device_common.cuh"

namespace cfsim {

namespace {

// A group of threads working on one pair: a single warp (bar < 0) or a set of
// whole warps synchronised by named barrier `bar`.  sum() contains the
// group's one barrier; `redf`/`redi` hold two parities of per-warp partials
// (2 * size / 32 entries) so that consecutive sums need no second barrier.
struct Group {
  int rank, size, bar;
  float* redf;
  int* redi;
  __device__ __forceinline__ int warp() const { return rank >> 5; }
  __device__ __forceinline__ int nwarps() const { return size >> 5; }
  __device__ __forceinline__ void sync() const {
    if (bar < 0)
      __syncwarp();
    else
      bar_sync(bar, size);
  }
  // Each warp writes its partial, then every warp reads all partials (one per
  // lane) and reduces them with the same butterfly, so all threads get the
  // same bits.
  __device__ __forceinline__ float sum(float v, int par) const {
    v = warp_sum(v);
    if (bar < 0) {
      __syncwarp();
      return v;
    }
    const int lane = rank & 31;
    if (lane == 0) redf[par * (size >> 5) + (rank >> 5)] = v;
    bar_sync(bar, size);
    return warp_sum(lane < (size >> 5) ? redf[par * (size >> 5) + lane] : 0.f);
  }
  __device__ __forceinline__ int sum_i(int v, int par) const {
    v = warp_sum_i(v);
    if (bar < 0) {
      __syncwarp();
      return v;
    }
    const int lane = rank & 31;
    if (lane == 0) redi[par * (size >> 5) + (rank >> 5)] = v;
    bar_sync(bar, size);
    return warp_sum_i(lane < (size >> 5) ? redi[par * (size >> 5) + lane] : 0);
  }
};

// Lists of one column-graph block j for the straight-line gather: its first
// two out- and in-neighbours as byte offsets v * 4 with weights, missing
// entries padded with {0, 0.0f}; flag != 0 when it has further neighbours
// (col_extra then reads their ranges from the staged row pointers).
struct ColPad {
  int vo0, vo1, vi0, vi1;
  float wo0, wo1, wi0, wi1;
  int flag;
};

// cptr = the column graph's staged row pointers (out: [0, n_col], in: after
// them, both local to its staged entries); cedge = its {v 4, w} entries.
__device__ __forceinline__ ColPad load_col(const int* cptr, const int2* cedge, int n_col, int j) {
  ColPad c;
  const int e0 = cptr[j], e1 = cptr[j + 1];
  int2 x = e1 > e0 ? cedge[e0] : make_int2(0, 0);
  c.vo0 = x.x;
  c.wo0 = __int_as_float(x.y);
  x = e1 > e0 + 1 ? cedge[e0 + 1] : make_int2(0, 0);
  c.vo1 = x.x;
  c.wo1 = __int_as_float(x.y);
  const int f0 = cptr[n_col + 1 + j], f1 = cptr[n_col + 2 + j];
  x = f1 > f0 ? cedge[f0] : make_int2(0, 0);
  c.vi0 = x.x;
  c.wi0 = __int_as_float(x.y);
  x = f1 > f0 + 1 ? cedge[f0 + 1] : make_int2(0, 0);
  c.vi1 = x.x;
  c.wi1 = __int_as_float(x.y);
  c.flag = (e1 - e0 > 2 || f1 - f0 > 2) ? 1 : 0;
  return c;
}

// Loads of the iterate at byte offset a + b: from a generic pointer (shared
// memory of this CTA, or global memory), or -- ClusterY -- from the
// distributed shared memory of a thread-block cluster, where a holds a 32-bit
// shared::cluster address (row u of the owning CTA's buffer 0) and the base
// the offset of the buffer being read.
struct ClusterY {
  uint32_t b;
};

__device__ __forceinline__ float lds_at(const char* base, int a, int b) {
  return *reinterpret_cast<const float*>(base + (a + b));
}

__device__ __forceinline__ float lds_at(ClusterY y, int a, int b) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(y.b + (uint32_t)a + (uint32_t)b));
  return v;
}

// Entry (i, j) of  sum_{i->u} sum_{j->v} w_iu w_jv Y[u,v] + sum_{u->i} sum_{v->j} w_ui w_vj Y[u,v]
// is split over the neighbour pairs as
//   (first two of i) x (first two of j)      gather_fast: straight-line, eight loads
// + (further ones of i) x (first two of j)   row_extra: same trip count for the lanes of row i
// + (all of i) x (further ones of j)         col_extra: only lanes whose column has them
// which covers every pair exactly once.  A = row i's first two out-neighbours
// {u ld 4, w} (the sign bit of A.w flags further neighbours of i), Q = its
// first two in-neighbours; padding entries carry weight 0.  (The cluster
// tier flags rows with a neighbour in another CTA by the sign bit of A.y.)
template <class YT>
__device__ __forceinline__ float gather_fast(YT Y, const int4 A, const int4 Q, const ColPad& c) {
  const float a0 = lds_at(Y, A.x, c.vo0), a1 = lds_at(Y, A.x, c.vo1);
  const float a2 = lds_at(Y, A.z, c.vo0), a3 = lds_at(Y, A.z, c.vo1);
  const float b0 = lds_at(Y, Q.x, c.vi0), b1 = lds_at(Y, Q.x, c.vi1);
  const float b2 = lds_at(Y, Q.z, c.vi0), b3 = lds_at(Y, Q.z, c.vi1);
  const float so = fmaf(fabsf(__int_as_float(A.w)), fmaf(c.wo1, a3, c.wo0 * a2),
                        fabsf(__int_as_float(A.y)) * fmaf(c.wo1, a1, c.wo0 * a0));
  const float si =
      fmaf(__int_as_float(Q.w), fmaf(c.wi1, b3, c.wi0 * b2), __int_as_float(Q.y) * fmaf(c.wi1, b1, c.wi0 * b0));
  return so + si;
}

// rr = row i's full out- and in-edge ranges into redge ({u ld 4, w}).
template <class YT>
__device__ __forceinline__ float row_extra(YT Y, const int4 rr, const int2* redge, const ColPad& c) {
  float s = 0.f;
  for (int k = rr.x + 2; k < rr.y; ++k) {
    const int2 e = redge[k];
    s = fmaf(__int_as_float(e.y), fmaf(c.wo1, lds_at(Y, e.x, c.vo1), c.wo0 * lds_at(Y, e.x, c.vo0)), s);
  }
  for (int k = rr.z + 2; k < rr.w; ++k) {
    const int2 e = redge[k];
    s = fmaf(__int_as_float(e.y), fmaf(c.wi1, lds_at(Y, e.x, c.vi1), c.wi0 * lds_at(Y, e.x, c.vi0)), s);
  }
  return s;
}

// cedge = the column graph's staged {v 4, w} entries (out-edges, then in-edges).
// cptr / n_col / j locate column j's further neighbours in cedge.
template <class YT>
__device__ __forceinline__ float col_extra(YT Y, const int4 A, const int4 Q, const int4 rr, const int2* redge,
                                           const int2* cedge, const int* cptr, int n_col, int j) {
  float s = 0.f;
  const int xo1 = cptr[j + 1], xi0 = cptr[n_col + 1 + j] + 2, xi1 = cptr[n_col + 2 + j];
  for (int f = cptr[j] + 2; f < xo1; ++f) {
    const int2 v = cedge[f];
    float t = fmaf(fabsf(__int_as_float(A.w)), lds_at(Y, A.z, v.x), fabsf(__int_as_float(A.y)) * lds_at(Y, A.x, v.x));
    for (int k = rr.x + 2; k < rr.y; ++k) {
      const int2 e = redge[k];
      t = fmaf(__int_as_float(e.y), lds_at(Y, e.x, v.x), t);
    }
    s = fmaf(__int_as_float(v.y), t, s);
  }
  for (int f = xi0; f < xi1; ++f) {
    const int2 v = cedge[f];
    float t = fmaf(__int_as_float(Q.w), lds_at(Y, Q.z, v.x), __int_as_float(Q.y) * lds_at(Y, Q.x, v.x));
    for (int k = rr.z + 2; k < rr.w; ++k) {
      const int2 e = redge[k];
      t = fmaf(__int_as_float(e.y), lds_at(Y, e.x, v.x), t);
    }
    s = fmaf(__int_as_float(v.y), t, s);
  }
  return s;
}

// Unit attribute vector of one block: a_f sqrt(omega_f) / r with
// r = sqrt(sum_f omega_f a_f^2), zero when r = 0, so that the cosine term of
// two blocks is the plain dot product of their unit vectors.  sq = sqrt(omega)
// (shared memory), Fp floats in and out.
__device__ __forceinline__ void unit_attr(const float* a, const float* sq, int Fp, float* out) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* s4 = reinterpret_cast<const float4*>(sq);
  float4* o4 = reinterpret_cast<float4*>(out);
  float acc = 0.f;
  for (int q = 0; q < (Fp >> 2); ++q) {
    const float4 v = __ldg(a4 + q), w = s4[q];
    const float4 u = make_float4(v.x * w.x, v.y * w.y, v.z * w.z, v.w * w.w);
    acc = fmaf(u.x, u.x, fmaf(u.y, u.y, fmaf(u.z, u.z, fmaf(u.w, u.w, acc))));
    o4[q] = u;
  }
  const float inv = acc > 0.f ? 1.0f / sqrtf(acc) : 0.f;
  for (int q = 0; q < (Fp >> 2); ++q) {
    const float4 u = o4[q];
    o4[q] = make_float4(u.x * inv, u.y * inv, u.z * inv, u.w * inv);
  }
}

// Shared state of the cluster kernel besides the pair region.
struct ClState {
  float part[2];       // this CTA's partial sum, two parities
  float redw[64];      // per-warp partials, two parities
  int parti[2];        // the same for integer sums
  int redwi[64];
  uint32_t q;          // the pair index CTA 0 pulled
  uint32_t rbase[kMaxCluster];  // cluster address of each CTA's region
  uint32_t paddr[kMaxCluster];  // cluster address of each CTA's part[]
  uint32_t piaddr[kMaxCluster]; // cluster address of each CTA's parti[]
  uint32_t qaddr;               // cluster address of CTA 0's q
  // the halo of a pair's slab (rows of other CTAs that its gathers read):
  // a bitmap over the row graph, its per-word prefix counts, the rows in
  // order, and this CTA's count / fit flag as the other CTAs read them
  uint32_t hbits[64];
  int hpre[64];
  int16_t hrow[512];
  int hcnt, hfit;
};
constexpr int kHaloRows = 512;   // halo rows a CTA may hold (hrow)
constexpr int kHaloMaxRows = 2048;  // row-graph size the halo bitmap covers

// Sum of v over every thread of the cluster, the same bits on every thread:
// warps -> CTA (one CTA barrier) -> cluster (one cluster barrier; lane r
// reads CTA r's partial).
__device__ __forceinline__ float cl_sum(float v, int par, ClState& st, int C) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) st.redw[par * 32 + w] = v;
  __syncthreads();
  if (w == 0) {
    const float x = warp_sum(lane < NW ? st.redw[par * 32 + lane] : 0.f);
    if (lane == 0) st.part[par] = x;
  }
  cl_sync();
  return warp_sum(lane < C ? cl_ld_f32(st.paddr[lane] + 4u * par) : 0.f);
}

__device__ __forceinline__ int cl_sum_i(int v, int par, ClState& st, int C) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
  v = warp_sum_i(v);
  if (lane == 0) st.redwi[par * 32 + w] = v;
  __syncthreads();
  if (w == 0) {
    const int x = warp_sum_i(lane < NW ? st.redwi[par * 32 + lane] : 0);
    if (lane == 0) st.parti[par] = x;
  }
  cl_sync();
  return warp_sum_i(lane < C ? (int)cl_ld_u32(st.piaddr[lane] + 4u * par) : 0);
}

// Every thread of a cluster as one group (the interface of Group): ranks and
// warps numbered across the CTAs, cluster barriers, cluster-wide sums.  The
// greedy matching runs on it with its state in global memory.
struct ClGroup {
  int rank, size, C;
  ClState* st;
  __device__ __forceinline__ int warp() const { return rank >> 5; }
  __device__ __forceinline__ int nwarps() const { return size >> 5; }
  __device__ __forceinline__ void sync() const { cl_sync(); }
  __device__ __forceinline__ float sum(float v, int par) const { return cl_sum(v, par, *st, C); }
  __device__ __forceinline__ int sum_i(int v, int par) const { return cl_sum_i(v, par, *st, C); }
};

}  // namespace

}  // namespace cfsim
