// The "best matching" alternative to greedy matching (Sec. 4.1 matches the
// nodes of two graphs; the optimal form maximises the summed similarity):
// a maximum-weight assignment of min(n_a, n_b) pairs on X_K, one warp per
// pair.
//
// Method: shortest augmenting paths with dual potentials (the Hungarian
// method in the Jonker-Volgenant formulation).  The smaller side gives the
// "rows"; costs are c(r, k) = xmax - x(r, k) >= 0, so minimising the summed
// cost maximises the summed similarity.  Rows are inserted one at a time; an
// insertion grows a Dijkstra tree over the columns on reduced costs
// c(r, k) - u(r) - v(k) until it reaches a free column, then flips the
// assignment along the tree path.  The columns are spread over the lanes
// (column k on lane k % 32).
//
// Two forms of one insertion:
//  - Up to 128 columns (every lane holds at most four): each lane keeps its
//    columns' potential v, owner row, tree distance and predecessor in
//    registers; the tree distances are absolute and the potentials move once
//    per insertion, after the free column is found (Crouse's rectangular
//    form), so a step is the relaxation of one cost row, a lane-local
//    minimum and two warp-wide unsigned minima (the distance, then the tie
//    rule: a free column first, then the smaller index).  Rows' u and the
//    row-to-column map sit in shared memory, and so does the whole X of a
//    pair where the warp's region holds it.
//  - Larger CFGs: the per-step form with every array in shared memory (the
//    potentials move by the step's minimum slack at every step).
//
// Work distribution (up to 128 columns): a CTA's first warps own large
// regions that hold the largest pair's X and take pairs from the front of
// the plan's queue (largest first); the other warps own small regions and
// take pairs from its back; both ends share one 64-bit counter, so every
// pair is taken exactly once.  A pair whose X does not fit the warp's region
// reads X from global memory.
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

constexpr int kOptNT = 1024;
constexpr size_t kOptSmem = 225280;
constexpr int kOptRegCols = 128;  // register form: at most four columns per lane

// ---- the register form ------------------------------------------------------

// Order-preserving map of a float to an unsigned key (negative values
// included) and its inverse.
__device__ __forceinline__ uint32_t ord_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_val(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Bytes of a warp region before its staged X: u and the row-to-column map
// for up to m_max rows.
__host__ __device__ __forceinline__ size_t opt_reg_head(int m_max) { return align_up(8 * (size_t)m_max, 16); }

// Bytes of a region that holds the X of any pair of up to m_max blocks a side.
__host__ __device__ __forceinline__ size_t opt_reg_big(int m_max) {
  return opt_reg_head(m_max) + align_up(4 * (size_t)m_max * m_max, 16);
}

// One pair on one warp, S = ceil(max(n_a, n_b) / 32) <= 4 columns per lane.
// X: n_a x n_b row-major (stride n_b).  Xs: room for the n x m cost rows in
// shared memory, or NULL to read X from global memory at every step.  u, c4r:
// n floats / ints of shared memory.  Writes match[n_a] (when mo is not NULL)
// and the score (every lane); returns false if an insertion found no finite
// reduced cost (NaN in X).
template <int S>
__device__ bool assign_regs(const float* __restrict__ X, int n_a, int n_b, float* __restrict__ Xs, float* u, int* c4r,
                            int32_t* mo, float* score) {
  const int lane = threadIdx.x & 31;
  const bool tr = n_a > n_b;  // rows = the smaller side
  const int n = tr ? n_b : n_a, m = tr ? n_a : n_b;
  float xmax = -CUDART_INF_F;
  if (Xs) {  // stage the n x m cost rows (x values; the cost is formed per step)
    int i = lane / (m > 0 ? m : 1), k = lane - i * m;
    for (int d = lane; d < n * m; d += 32) {
      const float x = __ldg(X + (tr ? (size_t)k * n_b + i : (size_t)i * n_b + k));
      Xs[d] = x;
      xmax = fmaxf(xmax, x);
      k += 32;
      while (k >= m) {
        k -= m;
        ++i;
      }
    }
  } else {
    for (size_t e = lane; e < (size_t)n_a * n_b; e += 32) xmax = fmaxf(xmax, __ldg(X + e));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  for (int i = lane; i < n; i += 32) {
    u[i] = 0.f;
    c4r[i] = -1;
  }
  float v[S];
  int own[S];
#pragma unroll
  for (int j = 0; j < S; ++j) {
    v[j] = 0.f;
    own[j] = -1;
  }
  __syncwarp();
  auto x_at = [&](int i, int k) -> float {
    return Xs ? Xs[i * m + k] : __ldg(X + (tr ? (size_t)k * n_b + i : (size_t)i * n_b + k));
  };
  bool ok = true;
  for (int cur = 0; cur < n; ++cur) {
    float spc[S];
    int path[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      spc[j] = CUDART_INF_F;
      path[j] = -1;
    }
    unsigned scanned = 0;
    float min_val = 0.f;
    int i = cur, sink = -1;
    for (int step = 0; step < m; ++step) {  // an insertion scans at most m columns
      const float ui = u[i];
      uint32_t kb = 0xffffffffu, ki = 0xffffffffu;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const int k = lane + 32 * j;
        if (k < m && !((scanned >> j) & 1u)) {
          const float r = min_val + ((xmax - x_at(i, k)) - ui - v[j]);
          if (r < spc[j]) {
            spc[j] = r;
            path[j] = i;
          }
          const uint32_t a = ord_key(spc[j]);
          const uint32_t b = (own[j] >= 0 ? 0x10000u : 0u) | (uint32_t)k;
          if (a < kb || (a == kb && b < ki)) {
            kb = a;
            ki = b;
          }
        }
      }
      const uint32_t wb = __reduce_min_sync(0xffffffffu, kb);
      const uint32_t wi = __reduce_min_sync(0xffffffffu, kb == wb ? ki : 0xffffffffu);
      if (wb >= ord_key(CUDART_INF_F)) break;  // no finite reduced cost left: X holds NaN
      min_val = key_val(wb);
      const int ks = (int)(wi & 0xffffu), wl = ks & 31, wj = ks >> 5;
      if (lane == wl) scanned |= 1u << wj;
      if (!(wi & 0x10000u)) {  // a free column: the path ends here
        sink = ks;
        break;
      }
      int o = -1;
#pragma unroll
      for (int j = 0; j < S; ++j)
        if (j == wj) o = own[j];
      i = __shfl_sync(0xffffffffu, o, wl);
    }
    if (sink < 0) {
      ok = false;
      break;
    }
    // move the potentials: every scanned column by its distance short of the
    // path's length, and its row (the owners; then the inserted row) to match
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if ((scanned >> j) & 1u) {
        const float dl = min_val - spc[j];
        v[j] -= dl;
        if (own[j] >= 0) u[own[j]] += dl;
      }
    }
    if (lane == 0) u[cur] += min_val;
    __syncwarp();
    // flip the assignment along the path from the free column back to row cur
    int j = sink;
    for (int hop = 0; hop <= n; ++hop) {
      const int jl = j & 31, jj = j >> 5;
      int pi = -1;
#pragma unroll
      for (int t = 0; t < S; ++t)
        if (t == jj) pi = path[t];
      pi = __shfl_sync(0xffffffffu, pi, jl);
      if (lane == jl) {
#pragma unroll
        for (int t = 0; t < S; ++t)
          if (t == jj) own[t] = pi;
      }
      const int prev = c4r[pi];
      __syncwarp();
      if (lane == 0) c4r[pi] = j;
      __syncwarp();
      if (pi == cur) break;
      j = prev;
    }
  }
  // the assignment in A's order, its value summed over the lanes
  float sc = 0.f;
  if (!tr) {
    for (int r = lane; r < n; r += 32) {
      const int k = c4r[r];
      if (mo) mo[r] = k;
      if (k >= 0) sc += __ldg(X + (size_t)r * n_b + k);
    }
  } else {
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const int k = lane + 32 * j;
      if (k < m) {
        if (mo) mo[k] = own[j];
        if (own[j] >= 0) sc += __ldg(X + (size_t)k * n_b + own[j]);
      }
    }
  }
  *score = warp_sum(sc);
  __syncwarp();
  return ok;
}

// ---- the per-step form (larger CFGs) ---------------------------------------

// Shared-memory bytes of one warp's state for up to m_max columns (and rows).
__host__ __device__ __forceinline__ size_t opt_warp_bytes(int m_max) { return align_up(25 * (size_t)(m_max + 1), 16); }

// Largest block count whose per-warp state fits the kernel's shared memory.
__host__ __device__ constexpr int opt_cap() { return (int)((kOptSmem - 16) / 25) - 1; }

// One pair on one warp (the per-step form).  X: n_a x n_b row-major (stride n_b).  Writes
// match[n_a] (when mo is not NULL) and the score (every lane); returns false
// if a step found no finite reduced cost (NaN in X).
__device__ bool assign_pair(const float* __restrict__ X, int n_a, int n_b, unsigned char* region, int32_t* mo,
                            float* score) {
  const int lane = threadIdx.x & 31;
  const bool tr = n_a > n_b;  // rows = the smaller side
  const int n = tr ? n_b : n_a, m = tr ? n_a : n_b;
  float* v = reinterpret_cast<float*>(region);
  float* minv = v + (m + 1);
  int32_t* way = reinterpret_cast<int32_t*>(minv + (m + 1));
  int32_t* owner = way + (m + 1);  // row assigned to column k, -1 none; index m is the tree root
  unsigned char* used = reinterpret_cast<unsigned char*>(owner + (m + 1));
  float* u = reinterpret_cast<float*>(region + align_up(17 * (size_t)(m + 1) + (size_t)(m + 1), 16));
  auto x_at = [&](int r, int k) -> float { return tr ? __ldg(X + (size_t)k * n_b + r) : __ldg(X + (size_t)r * n_b + k); };

  float xmax = -CUDART_INF_F;
  for (size_t e = lane; e < (size_t)n_a * n_b; e += 32) xmax = fmaxf(xmax, __ldg(X + e));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  for (int k = lane; k <= m; k += 32) {
    v[k] = 0.f;
    owner[k] = -1;
  }
  for (int r = lane; r < n; r += 32) u[r] = 0.f;
  __syncwarp();
  bool ok = true;
  for (int r = 0; r < n && ok; ++r) {
    // grow a shortest-path tree from row r, rooted at the virtual column m
    for (int k = lane; k < m; k += 32) {
      minv[k] = CUDART_INF_F;
      used[k] = 0;
    }
    if (lane == 0) {
      owner[m] = r;
      used[m] = 1;
    }
    __syncwarp();
    int cur = m;
    for (int steps = 0; steps <= m; ++steps) {
      const int i0 = owner[cur];
      const float ui = u[i0];
      float best = CUDART_INF_F;
      int bk = 0x7fffffff;
      for (int k = lane; k < m; k += 32) {
        if (used[k]) continue;
        const float red = (xmax - x_at(i0, k)) - ui - v[k];
        float mv = minv[k];
        if (red < mv) {
          mv = red;
          minv[k] = red;
          way[k] = cur;
        }
        if (mv < best) {  // lanes scan increasing k: ties keep the smaller column
          best = mv;
          bk = k;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        if (b2 < best || (b2 == best && k2 < bk)) {
          best = b2;
          bk = k2;
        }
      }
      if (bk == 0x7fffffff) {  // no finite reduced cost left: X holds NaN
        ok = false;
        break;
      }
      const float delta = best;
      // move the potentials: tree columns (and their rows) by delta, the
      // slack of the others down by delta
      for (int k = lane; k < m; k += 32) {
        if (used[k]) {
          u[owner[k]] += delta;
          v[k] -= delta;
        } else {
          minv[k] -= delta;
        }
      }
      if (lane == 0) {
        u[r] += delta;  // the root's row (owner[m])
        used[bk] = 1;
      }
      __syncwarp();
      cur = bk;
      if (owner[cur] < 0) break;  // reached a free column
    }
    if (!ok) break;
    // flip the assignment along the tree path back to the root
    if (lane == 0) {
      while (cur != m) {
        const int prev = way[cur];
        owner[cur] = owner[prev];
        cur = prev;
      }
    }
    __syncwarp();
  }
  // owner[k] = row of column k; report in A order with scores summed by column
  float sc = 0.f;
  if (!tr) {
    for (int i = lane; mo && i < n_a; i += 32) mo[i] = -1;
    __syncwarp();
    for (int k = lane; k < m; k += 32) {
      const int r = owner[k];
      if (r >= 0) {
        if (mo) mo[r] = k;
        sc += __ldg(X + (size_t)r * n_b + k);
      }
    }
  } else {
    for (int k = lane; k < m; k += 32) {
      const int r = owner[k];
      if (mo) mo[k] = r;
      if (r >= 0) sc += __ldg(X + (size_t)k * n_b + r);
    }
  }
  *score = warp_sum(sc);
  __syncwarp();
  return ok;
}

__device__ __forceinline__ int pack_max_blocks(const void* pack) {
  return reinterpret_cast<const PackHeader*>(pack)->max_blocks;
}

// Takes the next queue position from the front (or the back); -1 once the
// two ends have met.  One atomic on the 64-bit pair of counts orders every
// take, so a position is taken once.
__device__ __forceinline__ int take_pair(unsigned long long* ctr, bool front, uint32_t n_pairs) {
  const unsigned long long old = atomicAdd(ctr, front ? 1ull : (1ull << 32));
  const uint32_t f = (uint32_t)old, b = (uint32_t)(old >> 32);
  if ((uint64_t)f + b >= n_pairs) return -1;
  return front ? (int)f : (int)(n_pairs - 1 - b);
}

// Status and score of one finished pair.
__device__ __forceinline__ void finish_pair(const CallArgs& a, WsHeader* hdr, int p, bool ok, float sc) {
  if ((threadIdx.x & 31) == 0) {
    if (!ok) set_status(hdr, 6 /* CF_ERR_NUMERIC */, p);
    if (a.scores) a.scores[p] = sc;
  }
}

__global__ void __launch_bounds__(kOptNT) match_optimal_kernel(CallArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PackView A = load_pack(a.pack_a), B = load_pack(a.pack_b);
  const WsLayout L = ws_layout(a.P);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
  const uint32_t* queue = reinterpret_cast<const uint32_t*>(a.ws + L.queue);
  const int64_t* x_off = reinterpret_cast<const int64_t*>(a.ws + L.x_off);
  const int64_t* m_off = reinterpret_cast<const int64_t*>(a.ws + L.m_off);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(&hdr->q_opt);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_max = min(max(pack_max_blocks(a.pack_a), pack_max_blocks(a.pack_b)), opt_cap());
  uint32_t n_pairs = 0;
  for (int c = 0; c < kNumClasses; ++c) n_pairs += hdr->n_class[c];
  if (m_max <= kOptRegCols) {
    // warps [0, n_big): regions that hold any pair's X, front of the queue;
    // the others: equal shares of the rest, back of the queue
    const size_t bb = opt_reg_big(m_max);
    const int n_big = max(1, min(4, (int)(kOptSmem * 11 / 20 / bb)));
    const size_t bs = ((kOptSmem - (size_t)n_big * bb) / (kOptNT / 32 - n_big)) & ~(size_t)15;
    const bool big = w < n_big;
    unsigned char* region = big ? smem + (size_t)w * bb : smem + (size_t)n_big * bb + (size_t)(w - n_big) * bs;
    const size_t head = opt_reg_head(m_max);
    const size_t cap = ((big ? bb : bs) - head) / sizeof(float);
    float* u = reinterpret_cast<float*>(region);
    int* c4r = reinterpret_cast<int*>(u + m_max);
    float* xs = reinterpret_cast<float*>(region + head);
    for (;;) {
      int q = 0;
      if (lane == 0) q = take_pair(ctr, big, n_pairs);
      q = __shfl_sync(0xffffffffu, q, 0);
      if (q < 0) break;
      const int p = (int)queue[q];
      const int pa = a.pairs[2 * p], pb = a.pairs[2 * p + 1];
      const int na = A.node_off[pa + 1] - A.node_off[pa];
      const int nb = B.node_off[pb + 1] - B.node_off[pb];
      float* Xs = (size_t)na * nb <= cap ? xs : nullptr;
      const float* X = a.X_in + x_off[p];
      int32_t* mo = a.match ? a.match + m_off[p] : nullptr;
      float sc = 0.f;
      bool ok;
      switch ((max(na, nb) + 31) >> 5) {
        case 0:
        case 1: ok = assign_regs<1>(X, na, nb, Xs, u, c4r, mo, &sc); break;
        case 2: ok = assign_regs<2>(X, na, nb, Xs, u, c4r, mo, &sc); break;
        case 3: ok = assign_regs<3>(X, na, nb, Xs, u, c4r, mo, &sc); break;
        default: ok = assign_regs<4>(X, na, nb, Xs, u, c4r, mo, &sc); break;
      }
      finish_pair(a, hdr, p, ok, sc);
    }
    return;
  }
  // larger CFGs: the per-step form, regions sized for the larger pack's
  // largest CFG (capped at opt_cap()), front of the queue only
  int warps = (int)(kOptSmem / opt_warp_bytes(m_max));
  warps = warps > kOptNT / 32 ? kOptNT / 32 : warps;
  if (w >= warps) return;
  unsigned char* region = smem + (size_t)w * opt_warp_bytes(m_max);
  for (;;) {
    int q = 0;
    if (lane == 0) q = take_pair(ctr, true, n_pairs);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q < 0) break;
    const int p = (int)queue[q];
    const int pa = a.pairs[2 * p], pb = a.pairs[2 * p + 1];
    const int na = A.node_off[pa + 1] - A.node_off[pa];
    const int nb = B.node_off[pb + 1] - B.node_off[pb];
    if (na > m_max || nb > m_max) {  // a CFG above opt_cap() blocks
      if (lane == 0) set_status(hdr, 3 /* CF_ERR_UNSUPPORTED */, p);
      continue;
    }
    float sc = 0.f;
    int32_t* mo = a.match ? a.match + m_off[p] : nullptr;
    const bool ok = assign_pair(a.X_in + x_off[p], na, nb, region, mo, &sc);
    finish_pair(a, hdr, p, ok, sc);
  }
}

}  // namespace

int opt_max_blocks() { return opt_cap(); }

cudaError_t launch_match_optimal(const CallArgs& a, cudaStream_t s) {
  static bool init = false;
  static int grid = 0;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(match_optimal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOptSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    grid = n_sm;
    init = true;
  }
  const int g = a.P < grid ? a.P : grid;
  if (g > 0) match_optimal_kernel<<<g, kOptNT, kOptSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cfsim
