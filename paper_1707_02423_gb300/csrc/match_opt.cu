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
// Work distribution (up to 128 columns): every warp of a CTA draws its
// pair's X from a pool of 64 shared-memory slots under one 64-bit mask.
// Before it takes a pair from the plan's queue (largest pairs first), a
// warp reserves contiguous slots for the CTA's running estimate of the next
// pair's size (the size of the last pair a warp of the CTA took), then takes
// the pair and gives back the slots it does not need.  So no warp holds a
// pair it cannot stage, and waiting warps watch only the CTA's own mask
// (shared memory) for a release.  Every wait is bounded: past it a warp
// takes its pair and reads X from global memory instead.
#include "device_common.cuh"
#include "device_state.h"
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
  return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
}
__device__ __forceinline__ float key_val(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Bytes of a warp region before its staged X: u and the row-to-column map
// for up to m_max rows.
__host__ __device__ __forceinline__ size_t opt_reg_head(int m_max) { return align_up(8 * (size_t)m_max, 16); }

constexpr int kOptSlots = 64;           // shared-memory slots of the X pool (one 64-bit mask)
constexpr int kOptMaxWaits = 5000;      // polls of the slot mask before staging is given up (>= 10 ms)

// One pair on one warp, S = ceil(max(n_a, n_b) / 32) <= 4 columns per lane.
// X: n_a x n_b row-major (stride n_b).  kStaged: Xs holds room for the n x m
// cost rows in shared memory (else X is read from global memory at every
// step).  u, c4r: n floats / ints of shared memory.  Writes match[n_a] (when
// mo is not NULL) and the score (every lane); returns false if an insertion
// found no finite reduced cost (NaN in X).
template <int S, bool kStaged>
__device__ bool assign_regs(const float* __restrict__ X, int n_a, int n_b, float* __restrict__ Xs, float* u, int* c4r,
                            int32_t* mo, float* score) {
  const int lane = threadIdx.x & 31;
  const bool tr = n_a > n_b;  // rows = the smaller side
  const int n = tr ? n_b : n_a, m = tr ? n_a : n_b;
  float xmax = -CUDART_INF_F;
  if (kStaged) {
    // the n x m rows of x (the cost is formed per step): X read in its own
    // order (coalesced), eight loads in flight per lane, transposed into the
    // rows of the smaller side where n_a > n_b
    const int ne = n_a * n_b;
    for (int e0 = lane; e0 < ne; e0 += 32 * 8) {
      float xv[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) xv[t] = e0 + 32 * t < ne ? __ldg(X + e0 + 32 * t) : -CUDART_INF_F;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int e = e0 + 32 * t;
        if (e < ne) {
          const int ra = e / n_b, cb = e - ra * n_b;  // X(ra, cb)
          Xs[tr ? cb * m + ra : e] = xv[t];
          xmax = fmaxf(xmax, xv[t]);
        }
      }
    }
  } else {
#pragma unroll 8
    for (int e = lane; e < n_a * n_b; e += 32) xmax = fmaxf(xmax, __ldg(X + e));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  for (int i = lane; i < n; i += 32) {
    u[i] = 0.f;
    c4r[i] = -1;
  }
  // per column slot: potential, owner row, tie bits (owned flag << 16 | column)
  float v[S];
  int own[S], kc[S];
  uint32_t tb[S];
#pragma unroll
  for (int j = 0; j < S; ++j) {
    v[j] = 0.f;
    own[j] = -1;
    tb[j] = (uint32_t)(lane + 32 * j);
    kc[j] = min(lane + 32 * j, m - 1);  // in-range column for the loads of slots past m
  }
  __syncwarp();
  bool ok = true;
  for (int cur = 0; cur < n; ++cur) {
    float spc[S];
    int path[S];
    bool live[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      spc[j] = CUDART_INF_F;
      path[j] = -1;
      live[j] = lane + 32 * j < m;
    }
    float min_val = 0.f;
    int i = cur, sink = -1;
    for (int step = 0; step < m; ++step) {  // an insertion scans at most m columns
      const float ui = u[i];
      unsigned long long best = ~0ull;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const float x = kStaged ? Xs[i * m + kc[j]] : __ldg(X + (tr ? (size_t)kc[j] * n_b + i : (size_t)i * n_b + kc[j]));
        const float r = min_val + ((xmax - x) - ui - v[j]);
        const bool better = live[j] && r < spc[j];
        spc[j] = better ? r : spc[j];
        path[j] = better ? i : path[j];
        const uint32_t hi = live[j] ? ord_key(spc[j]) : 0xffffffffu;
        const unsigned long long key = ((unsigned long long)hi << 32) | tb[j];
        best = key < best ? key : best;
      }
      const uint32_t bh = (uint32_t)(best >> 32);
      const uint32_t wh = __reduce_min_sync(0xffffffffu, bh);
      const uint32_t wi = __reduce_min_sync(0xffffffffu, bh == wh ? (uint32_t)best : 0xffffffffu);
      if (wh >= ord_key(CUDART_INF_F)) break;  // no finite reduced cost left: X holds NaN
      min_val = key_val(wh);
      const int ks = (int)(wi & 0xffffu), wl = ks & 31, wj = ks >> 5;
      int o = own[0];
#pragma unroll
      for (int j = 1; j < S; ++j) o = wj == j ? own[j] : o;
#pragma unroll
      for (int j = 0; j < S; ++j) live[j] = live[j] && !(lane == wl && wj == j);
      if (!(wi & 0x10000u)) {  // a free column: the path ends here
        sink = ks;
        break;
      }
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
      if (lane + 32 * j < m && !live[j]) {
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
      int pi = path[0];
#pragma unroll
      for (int t = 1; t < S; ++t) pi = jj == t ? path[t] : pi;
      pi = __shfl_sync(0xffffffffu, pi, jl);
      if (lane == jl) {
#pragma unroll
        for (int t = 0; t < S; ++t) {
          if (t == jj) {
            own[t] = pi;
            tb[t] = 0x10000u | (uint32_t)(lane + 32 * t);
          }
        }
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

// Takes the next queue position; -1 once the queue is drained.
__device__ __forceinline__ int take_pair(unsigned long long* ctr, uint32_t n_pairs) {
  const unsigned long long old = atomicAdd(ctr, 1ull);
  return old < n_pairs ? (int)old : -1;
}

// Status and score of one finished pair.
__device__ __forceinline__ void finish_pair(const CallArgs& a, WsHeader* hdr, int p, bool ok, float sc) {
  if ((threadIdx.x & 31) == 0) {
    if (!ok) set_status(hdr, 6 /* CF_ERR_NUMERIC */, p);
    if (a.scores) a.scores[p] = sc;
  }
}

// First of k contiguous free slots in mask m; -1 if no run of k is free.
__device__ __forceinline__ int first_run(unsigned long long m, int k) {
  const unsigned long long fr = ~m;
  unsigned long long r = fr;  // bit s: slots s .. s + k - 1 all free
  for (int i = 1; i < k && r; ++i) r &= fr >> i;
  return r ? __ffsll((long long)r) - 1 : -1;
}

__device__ __forceinline__ unsigned long long run_bits(int s, int k) {
  return (k >= 64 ? ~0ull : ((1ull << k) - 1)) << s;
}

// Frees what wait_slots took, after the warp's last use of the slots.
__device__ __forceinline__ void release_slots(unsigned long long* mask, int s, int k) {
  __threadfence_block();
  atomicAnd(mask, ~run_bits(s, k));
}

// Takes k contiguous slots, waiting while other warps of the CTA hold them:
// a warp sleeps only while the mask still holds the very value in which it
// found no free run, so a release cannot go unseen.  -1 after max_polls
// polls (kOptMaxWaits; 0 under CF_FLAG_OPT_UNSTAGED) or if k can never fit.
__device__ __forceinline__ int wait_slots(unsigned long long* mask, int k, int max_polls) {
  if (k <= 0 || k > kOptSlots) return -1;
  for (int polls = 0; polls < max_polls; ++polls) {
    const unsigned long long m = *reinterpret_cast<volatile unsigned long long*>(mask);
    const int s = first_run(m, k);
    if (s >= 0) {
      if (atomicCAS(mask, m, m | run_bits(s, k)) == m) return s;
      continue;  // the mask moved under us: look again at once
    }
    while (polls < max_polls && *reinterpret_cast<volatile unsigned long long*>(mask) == m) {
      __nanosleep(4000);  // long sleeps: waiting warps must not take issue slots from working ones
      ++polls;
    }
  }
  return -1;
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
  const int max_polls = a.opt_unstaged ? 0 : kOptMaxWaits;
  uint32_t n_pairs = 0;
  for (int c = 0; c < kNumClasses; ++c) n_pairs += hdr->n_class[c];
  if (m_max <= kOptRegCols) {
    // per warp: u and the row-to-column map; then the X pool, kOptSlots
    // slots of `slot` bytes
    __shared__ unsigned long long s_mask;
    __shared__ int s_kest;
    const size_t head = opt_reg_head(m_max);
    const size_t slot = ((kOptSmem - (kOptNT / 32) * head) / kOptSlots) & ~(size_t)15;
    if (threadIdx.x == 0) {
      s_mask = 0ull;
      s_kest = (int)((4 * (size_t)m_max * m_max + slot - 1) / slot);
    }
    __syncthreads();
    unsigned char* pool = smem + (kOptNT / 32) * head;
    float* u = reinterpret_cast<float*>(smem + (size_t)w * head);
    int* c4r = reinterpret_cast<int*>(u + m_max);
    for (;;) {
      int q = -1, s0 = -1, k = 0;
      if (lane == 0) {
        // reserve room for the estimate, take a pair, keep what it needs
        const int k_est = *reinterpret_cast<volatile int*>(&s_kest);
        int r0 = wait_slots(&s_mask, k_est, max_polls);
        q = take_pair(ctr, n_pairs);
        if (q >= 0) {
          const int p = (int)queue[q];
          const int pa = a.pairs[2 * p], pb = a.pairs[2 * p + 1];
          const size_t bytes = 4 * (size_t)(A.node_off[pa + 1] - A.node_off[pa]) *
                               (size_t)(B.node_off[pb + 1] - B.node_off[pb]);
          k = (int)((bytes + slot - 1) / slot);
          s_kest = k > 0 ? k : 1;
          if (r0 >= 0 && k <= k_est) {
            if (k < k_est) release_slots(&s_mask, r0 + k, k_est - k);
            s0 = k > 0 ? r0 : -1;
          } else {
            if (r0 >= 0) release_slots(&s_mask, r0, k_est);
            s0 = k > 0 ? wait_slots(&s_mask, k, max_polls) : -1;
          }
        } else if (r0 >= 0) {
          release_slots(&s_mask, r0, k_est);
        }
      }
      q = __shfl_sync(0xffffffffu, q, 0);
      if (q < 0) break;
      s0 = __shfl_sync(0xffffffffu, s0, 0);
      k = __shfl_sync(0xffffffffu, k, 0);
      const int p = (int)queue[q];
      const int pa = a.pairs[2 * p], pb = a.pairs[2 * p + 1];
      const int na = A.node_off[pa + 1] - A.node_off[pa];
      const int nb = B.node_off[pb + 1] - B.node_off[pb];
      float* Xs = s0 >= 0 ? reinterpret_cast<float*>(pool + (size_t)s0 * slot) : nullptr;
      const float* X = a.X_in + x_off[p];
      int32_t* mo = a.match ? a.match + m_off[p] : nullptr;
      float sc = 0.f;
      const bool ok = Xs ? assign_regs<4, true>(X, na, nb, Xs, u, c4r, mo, &sc)
                         : assign_regs<4, false>(X, na, nb, Xs, u, c4r, mo, &sc);
      if (lane == 0 && s0 >= 0) release_slots(&s_mask, s0, k);  // assign_regs ends in a warp barrier
      finish_pair(a, hdr, p, ok, sc);
    }
    return;
  }
  // larger CFGs: the per-step form, regions sized for the larger pack's
  // largest CFG (capped at opt_cap())
  int warps = (int)(kOptSmem / opt_warp_bytes(m_max));
  warps = warps > kOptNT / 32 ? kOptNT / 32 : warps;
  if (w >= warps) return;
  unsigned char* region = smem + (size_t)w * opt_warp_bytes(m_max);
  for (;;) {
    int q = 0;
    if (lane == 0) q = take_pair(ctr, n_pairs);
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
  static DeviceOnce once;
  static int grids[kMaxDevices];
  int dev = 0;
  const cudaError_t ie = once.run(
      [](int d) {
        grids[d] = sm_count_of(d);
        return cudaFuncSetAttribute(match_optimal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOptSmem);
      },
      &dev);
  if (ie != cudaSuccess) return ie;
  const int grid = grids[dev];
  const int g = a.P < grid ? a.P : grid;
  if (g > 0) match_optimal_kernel<<<g, kOptNT, kOptSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cfsim
