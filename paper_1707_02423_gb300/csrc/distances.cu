// The paper's element-wise CFG distances (Sec. 4, 4.1, Table 1): the smaller
// CFG's transition matrix is resized by bilinear interpolation to the larger
// one's size, then Euclidean, Manhattan, Minkowski(p), Jaccard and Cosine
// distances are taken between the two N x N matrices; optionally each
// distance is min-max scaled to [0, 1] over all pairs of the call (Sec. 5.2).
//
// One warp per pair, pairs pulled from a counter.  The interpolated matrix is
// never stored: for output row r the warp scatters the two source rows it
// blends into a dense row buffer of n floats (shared memory), the larger
// graph's row r into a buffer of N floats, and every lane then forms x(r, c)
// and y(r, c) for its columns and accumulates |x - y|, |x - y|^2, |x - y|^p,
// x^2, y^2 and x y directly (no cancellation), in float within a row and in
// double across rows.  Sampling grid (corner-keeping): output index t samples
// the source at t (n - 1) / (N - 1).
#include <cmath>
#include <cstdio>

#include "../../include/cfsim.h"
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

constexpr int kDistNT = 512;
constexpr size_t kDistSmem = 225280;

struct DistWs {
  int32_t status, status_info;
  uint32_t q;
  uint32_t pad;
  uint32_t lo[kNumDist], hi[kNumDist];  // min / max of each distance (float bits, all values >= 0)
};

__host__ __device__ __forceinline__ size_t dist_warp_bytes(int m_max) { return align_up(8 * (size_t)(m_max + 1), 16); }

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

__global__ void __launch_bounds__(kDistNT) distances_kernel(const void* pack_a, const void* pack_b, const int32_t* pairs,
                                                           int P, float p, float* out, DistWs* ws) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PackView A = load_pack(pack_a), B = load_pack(pack_b);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_max = max(reinterpret_cast<const PackHeader*>(pack_a)->max_blocks,
                        reinterpret_cast<const PackHeader*>(pack_b)->max_blocks);
  const int warps = min((int)(kDistSmem / dist_warp_bytes(m_max)), kDistNT / 32);
  if (warps == 0) {  // a CFG above dist_max_blocks() blocks
    if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(&ws->status, 0, 3 /* CF_ERR_UNSUPPORTED */) == 0)
      ws->status_info = m_max;
    return;
  }
  if (w >= warps) return;
  float* R = reinterpret_cast<float*>(smem + (size_t)w * dist_warp_bytes(m_max));  // interpolated source row
  float* Y = R + (m_max + 1);                                                       // larger graph's row
  for (int k = lane; k <= m_max; k += 32) {
    R[k] = 0.f;
    Y[k] = 0.f;
  }
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
    double t_d2 = 0, t_d1 = 0, t_dp = 0, t_xx = 0, t_yy = 0, t_xy = 0;
    for (int r = 0; r < N; ++r) {
      int i0;
      float ar;
      grid_at(r, n, N, i0, ar);
      // R = (1 - ar) T_small[i0, :] + ar T_small[i0 + 1, :] (distinct columns within a row)
      const int e0 = S.out_ptr[sb + i0], e1 = S.out_ptr[sb + i0 + 1];
      for (int e = e0 + lane; e < e1; e += 32) {
        const CfAdj x = ldg_adj(S.out_adj + e);
        R[x.nbr] = (1.f - ar) * x.w;
      }
      __syncwarp();
      int f0 = 0, f1 = 0;
      if (ar != 0.f) {
        f0 = S.out_ptr[sb + i0 + 1];
        f1 = S.out_ptr[sb + i0 + 2];
        for (int e = f0 + lane; e < f1; e += 32) {
          const CfAdj x = ldg_adj(S.out_adj + e);
          R[x.nbr] += ar * x.w;
        }
      }
      const int g0 = L.out_ptr[lb + r], g1 = L.out_ptr[lb + r + 1];
      for (int e = g0 + lane; e < g1; e += 32) {
        const CfAdj y = ldg_adj(L.out_adj + e);
        Y[y.nbr] = y.w;
      }
      __syncwarp();
      float d2 = 0.f, d1 = 0.f, dp = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
      for (int c = lane; c < N; c += 32) {
        int j0;
        float bc;
        grid_at(c, n, N, j0, bc);
        const float x = bc != 0.f ? fmaf(bc, R[j0 + 1], (1.f - bc) * R[j0]) : R[j0];
        const float y = Y[c];
        const float d = fabsf(x - y);
        d2 = fmaf(d, d, d2);
        d1 += d;
        dp += powp(d, p);
        xx = fmaf(x, x, xx);
        yy = fmaf(y, y, yy);
        xy = fmaf(x, y, xy);
      }
      t_d2 += d2;
      t_d1 += d1;
      t_dp += dp;
      t_xx += xx;
      t_yy += yy;
      t_xy += xy;
      __syncwarp();
      // clear what this row wrote
      for (int e = e0 + lane; e < e1; e += 32) R[__ldg(&S.out_adj[e].nbr)] = 0.f;
      for (int e = f0 + lane; e < f1; e += 32) R[__ldg(&S.out_adj[e].nbr)] = 0.f;
      for (int e = g0 + lane; e < g1; e += 32) Y[__ldg(&L.out_adj[e].nbr)] = 0.f;
      __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t_d2 += __shfl_xor_sync(0xffffffffu, t_d2, o);
      t_d1 += __shfl_xor_sync(0xffffffffu, t_d1, o);
      t_dp += __shfl_xor_sync(0xffffffffu, t_dp, o);
      t_xx += __shfl_xor_sync(0xffffffffu, t_xx, o);
      t_yy += __shfl_xor_sync(0xffffffffu, t_yy, o);
      t_xy += __shfl_xor_sync(0xffffffffu, t_xy, o);
    }
    if (lane == 0) {
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

// Min-max scaling of each distance over the call's pairs (one CTA).
__global__ void __launch_bounds__(1024) distances_scale_kernel(int P, float* out, const DistWs* ws) {
  __shared__ float lo[kNumDist], span[kNumDist];
  if (threadIdx.x < kNumDist) {
    lo[threadIdx.x] = __uint_as_float(ws->lo[threadIdx.x]);
    span[threadIdx.x] = __uint_as_float(ws->hi[threadIdx.x]) - lo[threadIdx.x];
  }
  __syncthreads();
  for (size_t e = threadIdx.x; e < (size_t)P * kNumDist; e += blockDim.x) {
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
  while (dist_warp_bytes(m + 1) <= kDistSmem) ++m;
  return m;
}

cudaError_t launch_distances(const void* pack_a, const void* pack_b, const int32_t* pairs, int P, float p, bool scale,
                             float* out, void* ws, cudaStream_t s) {
  static bool init = false;
  static int grid = 0;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(distances_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDistSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    grid = n_sm;
    init = true;
  }
  DistWs* w = static_cast<DistWs*>(ws);
  distances_init_kernel<<<1, 32, 0, s>>>(w);
  const int g = P < grid ? P : grid;
  if (g > 0) distances_kernel<<<g, kDistNT, kDistSmem, s>>>(pack_a, pack_b, pairs, P, p, out, w);
  if (scale && P > 0) distances_scale_kernel<<<1, 1024, 0, s>>>(P, out, w);
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
