// Ward clustering of CFGs by their similarity profiles (Sec. 5.3: Ward's
// minimum-variance method on squared Euclidean distances), and the scatter of
// pair scores into the dense score matrix whose rows are those profiles.
//
// ward_dist_kernel: D[i][j] = |X_i - X_j|^2 for all point pairs (one thread
// per entry, D[i][i] = +inf).
// ward_merge_kernel (one CTA): n - 1 merges.  Each step takes the active pair
// (a < b) of smallest D (ties: smaller a, then smaller b) from a per-row
// minimum cache, records it in scipy's linkage convention (cluster ids, height
// sqrt(D), size), keeps the union in slot a and retires slot b, and updates
// row / column a by the Lance-Williams recurrence for Ward,
//   D(a u b, k) = ((n_a + n_k) D(a, k) + (n_b + n_k) D(b, k) - n_k D(a, b))
//                 / (n_a + n_b + n_k).
// Rows whose cached minimum pointed at a or b are rescanned (a warp each);
// the others only compare against their new entry for a.
#include <algorithm>
#include <cstdio>

#include "../../include/cfsim.h"
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

void set_error_detail(const char* msg);

namespace {

constexpr int kWardNT = 1024;

struct WardLayout {
  size_t hdr, D, size, active, rmin, rarg, cid, flag, total;
};

WardLayout ward_layout(int n) {
  WardLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = align_up(o + b, kAlign);
    return at;
  };
  L.hdr = take(64);
  L.D = take(4 * (size_t)n * n);
  L.size = take(4 * (size_t)n);
  L.active = take(4 * (size_t)n);
  L.rmin = take(4 * (size_t)n);
  L.rarg = take(4 * (size_t)n);
  L.cid = take(4 * (size_t)n);
  L.flag = take(4 * (size_t)n);
  L.total = o;
  return L;
}

struct WardPtrs {
  int32_t* hdr;  // status, status_info
  float* D;
  int32_t* size;
  int32_t* active;
  float* rmin;
  int32_t* rarg;
  int32_t* cid;
  int32_t* flag;
};

__global__ void ward_dist_kernel(const float* __restrict__ X, int n, int dim, float* __restrict__ D) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (i == j) {
    D[e] = CUDART_INF_F;
    return;
  }
  const float* xi = X + (size_t)i * dim;
  const float* xj = X + (size_t)j * dim;
  float s = 0.f;
  for (int k = 0; k < dim; ++k) {
    const float d = __ldg(xi + k) - __ldg(xj + k);
    s = fmaf(d, d, s);
  }
  D[e] = s;
}

// (value, a, b) lexicographic minimum.
__device__ __forceinline__ bool better(float v, int a, int b, float v2, int a2, int b2) {
  return v2 < v || (v2 == v && (a2 < a || (a2 == a && b2 < b)));
}

// Row minimum of active columns j != i (ties: smaller j), by one warp.
__device__ __forceinline__ void warp_row_min(const WardPtrs& w, int n, int i, float& bv, int& bj) {
  const int lane = threadIdx.x & 31;
  bv = CUDART_INF_F;
  bj = 0x7fffffff;
  const float* row = w.D + (size_t)i * n;
  for (int j = lane; j < n; j += 32) {
    if (j == i || !w.active[j]) continue;
    const float v = row[j];
    if (v < bv) {  // lanes scan increasing j: ties keep the smaller column
      bv = v;
      bj = j;
    }
  }
  warp_argmin(bv, bj);
}

__global__ void __launch_bounds__(kWardNT) ward_merge_kernel(WardPtrs w, int n, int32_t* merge, float* height,
                                                            int32_t* size_out) {
  __shared__ float s_v[32];
  __shared__ int s_a[32], s_b[32];
  __shared__ int s_pick[2];
  __shared__ float s_dab;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, NW = kWardNT / 32;
  for (int i = t; i < n; i += kWardNT) {
    w.size[i] = 1;
    w.active[i] = 1;
    w.cid[i] = i;
  }
  __syncthreads();
  for (int i = wid; i < n; i += NW) {
    float v;
    int j;
    warp_row_min(w, n, i, v, j);
    if (lane == 0) {
      w.rmin[i] = v;
      w.rarg[i] = j == 0x7fffffff ? -1 : j;
    }
  }
  __syncthreads();
  for (int step = 0; step < n - 1; ++step) {
    // (a) the closest active pair
    float bv = CUDART_INF_F;
    int ba = 0x7fffffff, bb = 0x7fffffff;
    for (int i = t; i < n; i += kWardNT) {
      if (!w.active[i] || w.rarg[i] < 0) continue;
      const int j = w.rarg[i];
      const int a = min(i, j), b = max(i, j);
      if (better(bv, ba, bb, w.rmin[i], a, b)) {
        bv = w.rmin[i];
        ba = a;
        bb = b;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int a2 = __shfl_xor_sync(0xffffffffu, ba, o), b2 = __shfl_xor_sync(0xffffffffu, bb, o);
      if (better(bv, ba, bb, v2, a2, b2)) {
        bv = v2;
        ba = a2;
        bb = b2;
      }
    }
    if (lane == 0) {
      s_v[wid] = bv;
      s_a[wid] = ba;
      s_b[wid] = bb;
    }
    __syncthreads();
    if (wid == 0) {
      bv = s_v[lane];
      ba = s_a[lane];
      bb = s_b[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int a2 = __shfl_xor_sync(0xffffffffu, ba, o), b2 = __shfl_xor_sync(0xffffffffu, bb, o);
        if (better(bv, ba, bb, v2, a2, b2)) {
          bv = v2;
          ba = a2;
          bb = b2;
        }
      }
      if (lane == 0) {
        s_pick[0] = ba;
        s_pick[1] = bb;
        s_dab = bv;
      }
    }
    __syncthreads();
    const int a = s_pick[0], b = s_pick[1];
    if (a == 0x7fffffff || !(s_dab < CUDART_INF_F)) {  // no finite distance left: NaN in the points
      if (t == 0 && atomicCAS(&w.hdr[0], 0, 6 /* CF_ERR_NUMERIC */) == 0) w.hdr[1] = step;
      return;
    }
    const float dab = s_dab;
    const int na = w.size[a], nb = w.size[b];
    if (t == 0) {
      const int ca = w.cid[a], cb = w.cid[b];
      merge[2 * step] = min(ca, cb);
      merge[2 * step + 1] = max(ca, cb);
      height[step] = sqrtf(fmaxf(dab, 0.f));
      size_out[step] = na + nb;
    }
    __syncthreads();
    // (c) Lance-Williams update of row / column a; retire b
    for (int k = t; k < n; k += kWardNT) {
      w.flag[k] = 0;
      if (k == a || k == b || !w.active[k]) continue;
      const float nk = (float)w.size[k];
      const float dak = w.D[(size_t)a * n + k], dbk = w.D[(size_t)b * n + k];
      const float v = (((float)na + nk) * dak + ((float)nb + nk) * dbk - nk * dab) / ((float)(na + nb) + nk);
      w.D[(size_t)a * n + k] = v;
      w.D[(size_t)k * n + a] = v;
      const int rk = w.rarg[k];
      if (rk == a || rk == b) {
        w.flag[k] = 1;  // its cached minimum may have moved: rescan
      } else if (v < w.rmin[k] || (v == w.rmin[k] && a < rk)) {
        w.rmin[k] = v;
        w.rarg[k] = a;
      }
    }
    __syncthreads();
    if (t == 0) {
      w.active[b] = 0;
      w.size[a] = na + nb;
      w.cid[a] = n + step;
      w.flag[a] = 1;
    }
    __syncthreads();
    // (d) rescans, a warp per flagged row
    for (int i = wid; i < n; i += NW) {
      if (!w.flag[i] || !w.active[i]) continue;
      float v;
      int j;
      warp_row_min(w, n, i, v, j);
      if (lane == 0) {
        w.rmin[i] = v;
        w.rarg[i] = j == 0x7fffffff ? -1 : j;
      }
    }
    __syncthreads();
  }
}

// S[a][b] = score of pair (a, b), and S[b][a] when symmetric; S zeroed first.
__global__ void zero_kernel(float* S, size_t m) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) S[e] = 0.f;
}

__global__ void scatter_scores_kernel(const int32_t* pairs, const float* scores, int P, int n_rows, int n_cols,
                                      int symmetric, float* S, int32_t* bad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int a = pairs[2 * p], b = pairs[2 * p + 1];
  if (a < 0 || a >= n_rows || b < 0 || b >= n_cols || (symmetric && (b >= n_rows || a >= n_cols))) {
    atomicCAS(bad, 0, p + 1);
    return;
  }
  S[(size_t)a * n_cols + b] = scores[p];
  if (symmetric) S[(size_t)b * n_cols + a] = scores[p];
}

void set_err(const char* m) { set_error_detail(m); }

}  // namespace

}  // namespace cfsim

using namespace cfsim;

extern "C" {

cf_status cf_ward_ws_size(int32_t n, size_t* bytes) {
  if (!bytes || n < 1 || n > 16384) {
    set_err("cf_ward_ws_size: need 1 <= n <= 16384 and bytes");
    return CF_ERR_INVALID_ARG;
  }
  *bytes = ward_layout(n).total;
  set_err("");
  return CF_OK;
}

cf_status cf_ward(const float* d_points, int32_t n, int32_t dim, int32_t* d_merge, float* d_height, int32_t* d_size,
                  void* d_ws, size_t ws_bytes, cf_stream_t stream) {
  if (n < 1 || n > 16384 || dim < 1 || !d_points || !d_ws || (n > 1 && (!d_merge || !d_height || !d_size))) {
    set_err("cf_ward: need 1 <= n <= 16384, dim >= 1 and non-NULL buffers");
    return CF_ERR_INVALID_ARG;
  }
  const WardLayout L = ward_layout(n);
  if (ws_bytes < L.total) {
    set_err("cf_ward: workspace too small (see cf_ward_ws_size)");
    return CF_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(d_ws);
  WardPtrs w;
  w.hdr = reinterpret_cast<int32_t*>(base + L.hdr);
  w.D = reinterpret_cast<float*>(base + L.D);
  w.size = reinterpret_cast<int32_t*>(base + L.size);
  w.active = reinterpret_cast<int32_t*>(base + L.active);
  w.rmin = reinterpret_cast<float*>(base + L.rmin);
  w.rarg = reinterpret_cast<int32_t*>(base + L.rarg);
  w.cid = reinterpret_cast<int32_t*>(base + L.cid);
  w.flag = reinterpret_cast<int32_t*>(base + L.flag);
  cudaError_t e = cudaMemsetAsync(w.hdr, 0, 64, st);
  if (e == cudaSuccess && n > 1) {
    const size_t m = (size_t)n * n;
    ward_dist_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(d_points, n, dim, w.D);
    ward_merge_kernel<<<1, kWardNT, 0, st>>>(w, n, d_merge, d_height, d_size);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "cf_ward: %s", cudaGetErrorString(e));
    set_err(buf);
    return CF_ERR_CUDA;
  }
  set_err("");
  return CF_OK;
}

cf_status cf_score_matrix(const int32_t* d_pairs, const float* d_scores, int32_t P, int32_t n_rows, int32_t n_cols,
                          int32_t symmetric, float* d_S, int32_t* d_status, cf_stream_t stream) {
  if (P < 0 || n_rows < 1 || n_cols < 1 || !d_S || !d_status || (P > 0 && (!d_pairs || !d_scores)) ||
      (symmetric && n_rows != n_cols)) {
    set_err("cf_score_matrix: bad sizes or NULL buffer (symmetric needs n_rows == n_cols)");
    return CF_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t m = (size_t)n_rows * n_cols;
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) {
    zero_kernel<<<(unsigned)std::min<size_t>((m + 255) / 256, 4096), 256, 0, st>>>(d_S, m);
    if (P > 0) scatter_scores_kernel<<<(P + 255) / 256, 256, 0, st>>>(d_pairs, d_scores, P, n_rows, n_cols, symmetric, d_S, d_status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "cf_score_matrix: %s", cudaGetErrorString(e));
    set_err(buf);
    return CF_ERR_CUDA;
  }
  set_err("");
  return CF_OK;
}

}  // extern "C"
