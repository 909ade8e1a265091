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
// c(r, k) - u(r) - v(k), moving the potentials by the tree's minimum slack at
// every step until a free column is reached, then flips the assignment along
// the tree path.  The columns are spread over the lanes (column k on lane
// k % 32): the per-step relaxation, argmin and potential update are one pass
// of each lane over its columns plus a warp reduction, with no block
// barrier.  Per-warp state lives in shared memory: v, minv (float), way,
// owner (int32) and a used flag per column, u per row.
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

constexpr int kOptNT = 512;
constexpr size_t kOptSmem = 225280;

// Shared-memory bytes of one warp's state for up to m_max columns (and rows).
__host__ __device__ __forceinline__ size_t opt_warp_bytes(int m_max) { return align_up(25 * (size_t)(m_max + 1), 16); }

// Largest block count whose per-warp state fits the kernel's shared memory.
__host__ __device__ constexpr int opt_cap() { return (int)((kOptSmem - 16) / 25) - 1; }

// One pair on one warp.  X: n_a x n_b row-major (stride n_b).  Writes
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

// Per-warp regions are sized for the larger of the two packs' largest CFGs
// (capped at opt_cap()); warps beyond what fits stay idle.  The plan's queue
// (largest pairs first) is drained through the q_opt counter.
__global__ void __launch_bounds__(kOptNT) match_optimal_kernel(CallArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PackView A = load_pack(a.pack_a), B = load_pack(a.pack_b);
  const WsLayout L = ws_layout(a.P);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
  const uint32_t* queue = reinterpret_cast<const uint32_t*>(a.ws + L.queue);
  const int64_t* x_off = reinterpret_cast<const int64_t*>(a.ws + L.x_off);
  const int64_t* m_off = reinterpret_cast<const int64_t*>(a.ws + L.m_off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_max = min(max(pack_max_blocks(a.pack_a), pack_max_blocks(a.pack_b)), opt_cap());
  int warps = (int)(kOptSmem / opt_warp_bytes(m_max));
  warps = warps > kOptNT / 32 ? kOptNT / 32 : warps;
  if (w >= warps) return;
  unsigned char* region = smem + (size_t)w * opt_warp_bytes(m_max);
  uint32_t n_pairs = 0;
  for (int c = 0; c < kNumClasses; ++c) n_pairs += hdr->n_class[c];
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(&hdr->q_opt, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= n_pairs) break;
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
    if (!ok && lane == 0) set_status(hdr, 6 /* CF_ERR_NUMERIC */, p);
    if (a.scores && lane == 0) a.scores[p] = sc;
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
