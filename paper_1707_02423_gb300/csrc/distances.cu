// The paper's element-wise CFG distances (Sec. 4, 4.1, Table 1): the smaller
// CFG's transition matrix is resized by bilinear interpolation to the larger
// one's size, then Euclidean, Manhattan, Minkowski(p), Jaccard and Cosine
// distances are taken between the two N x N matrices; optionally each
// distance is min-max scaled to [0, 1] over all pairs of the call (Sec. 5.2).
//
// One warp per pair, 32 warps per CTA, pairs pulled from a counter.  The
// interpolated matrix is never stored: for output row r the warp blends the
// two source rows it samples into a dense row buffer of n floats (shared
// memory), scatters the larger graph's row r into a buffer of N floats, and
// every lane then forms x(r, c) and y(r, c) for its columns and accumulates
// |x - y|, |x - y|^2, |x - y|^p, x^2, y^2 and x y directly (no cancellation),
// in float within a row and in compensated float sums (about twice float
// precision) across rows; the 32 lanes' sums meet in double.  Sampling grid
// (corner-keeping): output index t samples the source at t (n - 1) / (N - 1).
//
// Small CFGs (the staged layout): the pair's CSR rows and the column grid sit
// in the warp's shared memory and the row buffers rotate over three copies,
// so a row costs one warp barrier and no global-memory round trip.  Larger
// CFGs (the lean layout) read the CSR from global memory with one buffer of
// each side.
#include <cmath>
#include <cstdio>

#include "../../include/cfsim.h"
#include "device_common.cuh"
#include "device_state.h"
#include "kernels.h"

namespace cfsim {

namespace {

constexpr int kDistNT = 1024;
constexpr size_t kDistSmem = 225280;
constexpr int kDistMinStagedEdges = 64;

struct DistWs {
  int32_t status, status_info;
  uint32_t q;
  uint32_t pad;
  uint32_t lo[kNumDist], hi[kNumDist];  // min / max of each distance (float bits, all values >= 0)
};

// Per-warp shared memory of the lean layout: one row buffer of each side.
__host__ __device__ __forceinline__ size_t dist_lean_bytes(int m_max) { return align_up(8 * (size_t)(m_max + 1), 16); }

// Per-warp shared memory of the staged layout before its edge area: three row
// buffers of each side, the column grid (j0, bc) and both CFGs' row pointers.
__host__ __device__ __forceinline__ size_t dist_staged_bytes(int m_max) {
  return align_up(24 * (size_t)(m_max + 1) + 8 * (size_t)(m_max + 1) + 8 * (size_t)(m_max + 2), 16);
}

// Source coordinate of output index t: i0 and the weight a of row i0 + 1.
__device__ __forceinline__ void grid_at(int t, int n, int N, int& i0, float& a) {
  if (n == 1 || N == 1) {
    i0 = 0;
    a = 0.f;
    return;
  }
  const float f = (float)((long long)t * (n - 1)) / (float)(N - 1);
  i0 = min((int)floorf(f), n - 2);
  a = f - (float)i0;
}

__device__ __forceinline__ float powp(float d, float p) {
  return p == 3.f ? d * d * d : p == 2.f ? d * d : p == 1.f ? d : powf(d, p);
}

// Compensated running sums (Knuth's TwoSum): h + l carries the sum of the
// added floats to about twice float precision.
struct Sums6 {
  float h[6], l[6];
};

__device__ __forceinline__ void two_sum_add(float& h, float& l, float v) {
  const float s = h + v;
  const float bp = s - h;
  l += (h - (s - bp)) + (v - bp);
  h = s;
}

// One output row's per-lane partials, added into the running sums.
__device__ __forceinline__ void add_row(Sums6& t, float d2, float d1, float dp, float xx, float yy, float xy) {
  two_sum_add(t.h[0], t.l[0], d2);
  two_sum_add(t.h[1], t.l[1], d1);
  two_sum_add(t.h[2], t.l[2], dp);
  two_sum_add(t.h[3], t.l[3], xx);
  two_sum_add(t.h[4], t.l[4], yy);
  two_sum_add(t.h[5], t.l[5], xy);
}

// The terms of one entry: x of the interpolated matrix, y of the larger one.
__device__ __forceinline__ void add_entry(float x, float y, float p, float& d2, float& d1, float& dp, float& xx,
                                          float& yy, float& xy) {
  const float d = fabsf(x - y);
  d2 = fmaf(d, d, d2);
  d1 += d;
  dp += powp(d, p);
  xx = fmaf(x, x, xx);
  yy = fmaf(y, y, yy);
  xy = fmaf(x, y, xy);
}

// The pair's CSR in the warp's shared memory: sp / lp row pointers of the
// smaller / larger CFG relative to their first edge, sa / la their edges.
// Output row r blends source rows i0 and i0 + 1 into R (shared-memory
// atomics: a column holds at most one entry of each source row, so the two
// products land on zero in either order with the same float result) and
// scatters the larger CFG's row r into Y.  The three buffers of each side
// rotate: the buffers read at row r - 1 are cleared at row r, one warp
// barrier before row r + 2 writes them again, so each row needs one barrier.
__device__ __forceinline__ void pair_rows_staged(int n, int N, float p, const int* sp, const CfAdj* sa, const int* lp,
                                                 const CfAdj* la, float* R, float* Y, int ld, const float2* G,
                                                 Sums6& t) {
  const int lane = threadIdx.x & 31;
  int b = 0;
  for (int r = 0; r < N; ++r) {
    float* Rb = R + b * ld;
    float* Yb = Y + b * ld;
    int i0;
    float ar;
    grid_at(r, n, N, i0, ar);
    const int e0 = sp[i0], e1 = sp[i0 + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
      const CfAdj x = sa[e];
      atomicAdd(Rb + x.nbr, (1.f - ar) * x.w);
    }
    if (ar != 0.f) {
      const int f1 = sp[i0 + 2];
      for (int e = e1 + lane; e < f1; e += 32) {
        const CfAdj x = sa[e];
        atomicAdd(Rb + x.nbr, ar * x.w);
      }
    }
    const int g0 = lp[r], g1 = lp[r + 1];
    for (int e = g0 + lane; e < g1; e += 32) {
      const CfAdj y = la[e];
      Yb[y.nbr] = y.w;
    }
    __syncwarp();
    float d2 = 0.f, d1 = 0.f, dp = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
    for (int c = lane; c < N; c += 32) {
      const float2 g = G[c];
      const int j0 = __float_as_int(g.x);
      const float bc = g.y;
      const float x = bc != 0.f ? fmaf(bc, Rb[j0 + 1], (1.f - bc) * Rb[j0]) : Rb[j0];
      add_entry(x, Yb[c], p, d2, d1, dp, xx, yy, xy);
    }
    add_row(t, d2, d1, dp, xx, yy, xy);
    // clear the buffers of row r - 1 (every reader of them passed this row's barrier)
    const int bz = b == 0 ? 2 : b - 1;
    for (int k = lane; k < n; k += 32) R[bz * ld + k] = 0.f;
    for (int c = lane; c < N; c += 32) Y[bz * ld + c] = 0.f;
    b = b == 2 ? 0 : b + 1;
  }
  // clear the last row's buffers (the one before it was cleared in the loop)
  __syncwarp();
  const int bl = (N - 1) % 3;
  for (int k = lane; k < n; k += 32) R[bl * ld + k] = 0.f;
  for (int c = lane; c < N; c += 32) Y[bl * ld + c] = 0.f;
  __syncwarp();
}

// The same rows with the CSR read from global memory and a single buffer of
// each side (CFGs too large for the staged layout, or pairs with more edges
// than its edge area holds): three warp barriers per row.
__device__ __forceinline__ void pair_rows_global(int n, int N, float p, const int32_t* sptr, const int32_t* lptr,
                                                 const CfAdj* sadj, const CfAdj* ladj, float* R, float* Y, Sums6& t) {
  const int lane = threadIdx.x & 31;
  for (int r = 0; r < N; ++r) {
    int i0;
    float ar;
    grid_at(r, n, N, i0, ar);
    const int e0 = __ldg(sptr + i0), e1 = __ldg(sptr + i0 + 1);
    const int f1 = ar != 0.f ? __ldg(sptr + i0 + 2) : e1;
    for (int e = e0 + lane; e < e1; e += 32) {
      const CfAdj x = ldg_adj(sadj + e);
      atomicAdd(R + x.nbr, (1.f - ar) * x.w);
    }
    for (int e = e1 + lane; e < f1; e += 32) {
      const CfAdj x = ldg_adj(sadj + e);
      atomicAdd(R + x.nbr, ar * x.w);
    }
    const int g0 = __ldg(lptr + r), g1 = __ldg(lptr + r + 1);
    for (int e = g0 + lane; e < g1; e += 32) {
      const CfAdj y = ldg_adj(ladj + e);
      Y[y.nbr] = y.w;
    }
    __syncwarp();
    float d2 = 0.f, d1 = 0.f, dp = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
    for (int c = lane; c < N; c += 32) {
      int j0;
      float bc;
      grid_at(c, n, N, j0, bc);
      const float x = bc != 0.f ? fmaf(bc, R[j0 + 1], (1.f - bc) * R[j0]) : R[j0];
      add_entry(x, Y[c], p, d2, d1, dp, xx, yy, xy);
    }
    add_row(t, d2, d1, dp, xx, yy, xy);
    __syncwarp();
    // clear what this row wrote
    for (int e = e0 + lane; e < f1; e += 32) R[__ldg(&sadj[e].nbr)] = 0.f;
    for (int e = g0 + lane; e < g1; e += 32) Y[__ldg(&ladj[e].nbr)] = 0.f;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kDistNT) distances_kernel(const void* pack_a, const void* pack_b, const int32_t* pairs,
                                                           int P, float p, float* out, DistWs* ws) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PackView A = load_pack(pack_a), B = load_pack(pack_b);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_max = max(reinterpret_cast<const PackHeader*>(pack_a)->max_blocks,
                        reinterpret_cast<const PackHeader*>(pack_b)->max_blocks);
  // staged layout when every warp of the CTA gets its buffers plus a useful
  // edge area; else the lean layout on as many warps as fit
  const size_t staged_region = (kDistSmem / (kDistNT / 32)) & ~(size_t)15;
  const bool staged = dist_staged_bytes(m_max) + 8 * (size_t)kDistMinStagedEdges <= staged_region;
  const size_t region = staged ? staged_region : dist_lean_bytes(m_max);
  const int warps = staged ? kDistNT / 32 : min((int)(kDistSmem / region), kDistNT / 32);
  if (warps == 0) {  // a CFG above dist_max_blocks() blocks
    if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(&ws->status, 0, 3 /* CF_ERR_UNSUPPORTED */) == 0)
      ws->status_info = m_max;
    return;
  }
  if (w >= warps) return;
  unsigned char* base = smem + (size_t)w * region;
  const int ld = m_max + 1;
  float* R = reinterpret_cast<float*>(base);  // staged: R[3][ld], Y[3][ld]; lean: R[ld], Y[ld]
  float* Y = R + (staged ? 3 : 1) * ld;
  float2* G = reinterpret_cast<float2*>(Y + 3 * ld);  // staged only
  int* sp = reinterpret_cast<int*>(G + ld);
  int* lp = sp + (m_max + 2);
  CfAdj* ea = reinterpret_cast<CfAdj*>(base + dist_staged_bytes(m_max));
  const int cap_e = staged ? (int)((region - dist_staged_bytes(m_max)) / sizeof(CfAdj)) : 0;
  for (int k = lane; k < (staged ? 6 : 2) * ld; k += 32) R[k] = 0.f;
  __syncwarp();
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(&ws->q, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= (uint32_t)P) break;
    const int pa = pairs[2 * q], pb = pairs[2 * q + 1];
    if (pa < 0 || pa >= A.n_cfgs || pb < 0 || pb >= B.n_cfgs) {
      if (lane == 0 && atomicCAS(&ws->status, 0, 1 /* CF_ERR_INVALID_ARG */) == 0) ws->status_info = (int)q;
      continue;
    }
    const int na = A.node_off[pa + 1] - A.node_off[pa], nb = B.node_off[pb + 1] - B.node_off[pb];
    const bool a_small = na <= nb;
    const PackView& S = a_small ? A : B;
    const PackView& L = a_small ? B : A;
    const int sb = a_small ? A.node_off[pa] : B.node_off[pb];
    const int lb = a_small ? B.node_off[pb] : A.node_off[pa];
    const int n = a_small ? na : nb, N = a_small ? nb : na;
    Sums6 t;
#pragma unroll
    for (int k = 0; k < 6; ++k) t.h[k] = t.l[k] = 0.f;
    const int s0 = __ldg(S.out_ptr + sb), l0 = __ldg(L.out_ptr + lb);
    const int es = __ldg(S.out_ptr + sb + n) - s0, el = __ldg(L.out_ptr + lb + N) - l0;
    if (staged && es + el <= cap_e) {
      for (int i = lane; i <= n; i += 32) sp[i] = __ldg(S.out_ptr + sb + i) - s0;
      for (int i = lane; i <= N; i += 32) lp[i] = __ldg(L.out_ptr + lb + i) - l0;
      for (int e = lane; e < es; e += 32) ea[e] = ldg_adj(S.out_adj + s0 + e);
      for (int e = lane; e < el; e += 32) ea[es + e] = ldg_adj(L.out_adj + l0 + e);
      for (int c = lane; c < N; c += 32) {  // read back by the same lane only
        int j0;
        float bc;
        grid_at(c, n, N, j0, bc);
        G[c] = make_float2(__int_as_float(j0), bc);
      }
      __syncwarp();
      pair_rows_staged(n, N, p, sp, ea, lp, ea + es, R, Y, ld, G, t);
    } else {
      pair_rows_global(n, N, p, S.out_ptr + sb, L.out_ptr + lb, S.out_adj, L.out_adj, R, Y, t);
    }
    double v6[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double v = (double)t.h[k] + (double)t.l[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      v6[k] = v;
    }
    if (lane == 0) {
      const double t_d2 = v6[0], t_d1 = v6[1], t_dp = v6[2], t_xx = v6[3], t_yy = v6[4], t_xy = v6[5];
      const double den = t_xx + t_yy - t_xy;
      const double nx = sqrt(t_xx), ny = sqrt(t_yy);
      float v[kNumDist];
      v[0] = (float)sqrt(t_d2);
      v[1] = (float)t_d1;
      v[2] = (float)pow(t_dp, 1.0 / (double)p);
      v[3] = den > 0 ? (float)(t_d2 / den) : 0.f;
      v[4] = (nx > 0 && ny > 0) ? (float)(1.0 - t_xy / (nx * ny)) : ((nx == 0 && ny == 0) ? 0.f : 1.f);
      for (int k = 0; k < kNumDist; ++k) {
        v[k] = fmaxf(v[k], 0.f);  // rounding can leave the cosine distance of identical matrices at -1 ulp
        out[(size_t)q * kNumDist + k] = v[k];
        atomicMin(&ws->lo[k], __float_as_uint(v[k]));
        atomicMax(&ws->hi[k], __float_as_uint(v[k]));
      }
    }
  }
}

// Min-max scaling of each distance over the call's pairs (grid-stride over
// the P x 5 values).
__global__ void __launch_bounds__(256) distances_scale_kernel(int P, float* out, const DistWs* ws) {
  __shared__ float lo[kNumDist], span[kNumDist];
  if (threadIdx.x < kNumDist) {
    lo[threadIdx.x] = __uint_as_float(ws->lo[threadIdx.x]);
    span[threadIdx.x] = __uint_as_float(ws->hi[threadIdx.x]) - lo[threadIdx.x];
  }
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)P * kNumDist;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % kNumDist);
    out[e] = span[k] > 0.f ? (out[e] - lo[k]) / span[k] : 0.f;
  }
}

__global__ void distances_init_kernel(DistWs* ws) {
  if (threadIdx.x == 0) {
    ws->status = 0;
    ws->status_info = 0;
    ws->q = 0;
  }
  if (threadIdx.x < kNumDist) {
    ws->lo[threadIdx.x] = 0x7f800000u;  // +inf
    ws->hi[threadIdx.x] = 0u;
  }
}

}  // namespace

size_t dist_ws_bytes() { return align_up(sizeof(DistWs), kAlign); }

int dist_max_blocks() {
  int m = 1;
  while (dist_lean_bytes(m + 1) <= kDistSmem) ++m;
  return m;
}

cudaError_t launch_distances(const void* pack_a, const void* pack_b, const int32_t* pairs, int P, float p, bool scale,
                             float* out, void* ws, cudaStream_t s) {
  static DeviceOnce once;
  static int grids[kMaxDevices];
  int dev = 0;
  const cudaError_t ie = once.run(
      [](int d) {
        grids[d] = sm_count_of(d);
        return cudaFuncSetAttribute(distances_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDistSmem);
      },
      &dev);
  if (ie != cudaSuccess) return ie;
  const int grid = grids[dev];
  DistWs* w = static_cast<DistWs*>(ws);
  distances_init_kernel<<<1, 32, 0, s>>>(w);
  const int g = P < grid ? P : grid;
  if (g > 0) distances_kernel<<<g, kDistNT, kDistSmem, s>>>(pack_a, pack_b, pairs, P, p, out, w);
  if (scale && P > 0) {
    const size_t blocks = ((size_t)P * kNumDist + 255) / 256;
    distances_scale_kernel<<<(unsigned)(blocks < (size_t)grid ? blocks : (size_t)grid), 256, 0, s>>>(P, out, w);
  }
  return cudaGetLastError();
}

}  // namespace cfsim

namespace cfsim {
void set_error_detail(const char* msg);
}

extern "C" {

cf_status cf_distances_ws_size(int32_t P, size_t* bytes) {
  if (!bytes || P < 0) {
    cfsim::set_error_detail("need P >= 0 and bytes");
    return CF_ERR_INVALID_ARG;
  }
  *bytes = cfsim::dist_ws_bytes();
  cfsim::set_error_detail("");
  return CF_OK;
}

cf_status cf_distances(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P, float p,
                       uint32_t flags, float* d_out, void* d_ws, size_t ws_bytes, cf_stream_t stream) {
  if (P < 0 || !d_pack_a || !d_pack_b || !d_ws || (P > 0 && (!d_pairs || !d_out))) {
    cfsim::set_error_detail("cf_distances: NULL buffer or P < 0");
    return CF_ERR_INVALID_ARG;
  }
  if (!(p > 0.f && p <= 64.f)) {
    cfsim::set_error_detail("cf_distances: the Minkowski order p must be in (0, 64]");
    return CF_ERR_INVALID_ARG;
  }
  if (flags & ~(uint32_t)CF_DIST_SCALE01) {
    cfsim::set_error_detail("cf_distances: unknown flags");
    return CF_ERR_INVALID_ARG;
  }
  if (ws_bytes < cfsim::dist_ws_bytes()) {
    cfsim::set_error_detail("cf_distances: workspace too small (see cf_distances_ws_size)");
    return CF_ERR_WORKSPACE;
  }
  const cudaError_t e = cfsim::launch_distances(d_pack_a, d_pack_b, d_pairs, P, p, (flags & CF_DIST_SCALE01) != 0,
                                                d_out, d_ws, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "cf_distances launch: %s", cudaGetErrorString(e));
    cfsim::set_error_detail(buf);
    return CF_ERR_CUDA;
  }
  cfsim::set_error_detail("");
  return CF_OK;
}

}  // extern "C"
