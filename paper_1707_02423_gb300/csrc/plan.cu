// a7 (batch scheduler), device side: validate the pair list, classify every
// pair into an execution class, order the pairs by cost (largest first, two
// buckets per octave) into one queue per class, and compute the output offsets
// x_off[p] = sum_{q<p} n_a n_b and m_off[p] = sum_{q<p} n_a.
//
// Three small launches: count (per-pair class/bucket histogram and per-block
// offset sums), scan (one CTA: bucket cursors and block offsets), scatter
// (queue positions and per-pair offsets).  No host round trip, so the whole
// call can be replayed from a CUDA graph.
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

struct PlanCtx {
  PackView A, B;
  int P;
  const int32_t* pairs;
  WsHeader* hdr;
  uint32_t* queue;
  int64_t* x_off;
  int64_t* m_off;
  int64_t* bsum;  // [2][plan_blocks]
  int nblk;
};

__device__ __forceinline__ PlanCtx plan_ctx(const CallArgs& a) {
  PlanCtx c;
  c.A = load_pack(a.pack_a);
  c.B = load_pack(a.pack_b);
  c.P = a.P;
  c.pairs = a.pairs;
  WsLayout L = ws_layout(a.P);
  c.hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
  c.queue = reinterpret_cast<uint32_t*>(a.ws + L.queue);
  c.x_off = reinterpret_cast<int64_t*>(a.ws + L.x_off);
  c.m_off = reinterpret_cast<int64_t*>(a.ws + L.m_off);
  c.bsum = reinterpret_cast<int64_t*>(a.ws + L.bsum);
  c.nblk = L.plan_blocks;
  return c;
}

struct PairFacts {
  bool valid;
  int na, nb, ea, eb;
  int cls, bucket;
  int n_row, ld;  // resident matrix shape (classify)
};

__device__ __forceinline__ PairFacts pair_facts(const PlanCtx& c, int p, const ClassCfg& cc) {
  PairFacts f{};
  int pa = __ldg(c.pairs + 2 * p), pb = __ldg(c.pairs + 2 * p + 1);
  f.valid = pa >= 0 && pa < c.A.n_cfgs && pb >= 0 && pb < c.B.n_cfgs;
  if (!f.valid) {
    f.cls = kClassSkip;
    return f;
  }
  f.na = __ldg(c.A.node_off + pa + 1) - __ldg(c.A.node_off + pa);
  f.nb = __ldg(c.B.node_off + pb + 1) - __ldg(c.B.node_off + pb);
  const int ea = __ldg(c.A.edge_off + pa + 1) - __ldg(c.A.edge_off + pa);
  const int eb = __ldg(c.B.edge_off + pb + 1) - __ldg(c.B.edge_off + pb);
  f.ea = ea;
  f.eb = eb;
  Shape s = classify(f.na, f.nb, ea, eb, cc, __ldg(c.A.xdeg + pa), __ldg(c.B.xdeg + pb));
  f.cls = s.cls;
  f.n_row = s.n_row;
  f.ld = s.ld;
  // per-iteration work: every entry is written once, every edge pair gathered twice
  f.bucket = cost_bucket((int64_t)f.na * f.nb + 2 * (int64_t)ea * eb);
  return f;
}

// Exclusive block scan of two int64 values (256 threads).
__device__ __forceinline__ void block_scan2(int64_t& x, int64_t& m, int64_t& tx, int64_t& tm) {
  __shared__ int64_t sx[kPlanThreads / 32], sm[kPlanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t ix = x, im = m;  // inclusive within warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t ux = __shfl_up_sync(0xffffffffu, ix, o);
    int64_t um = __shfl_up_sync(0xffffffffu, im, o);
    if (lane >= o) {
      ix += ux;
      im += um;
    }
  }
  if (lane == 31) {
    sx[w] = ix;
    sm[w] = im;
  }
  __syncthreads();
  int64_t bx = 0, bm = 0;
  tx = 0;
  tm = 0;
#pragma unroll
  for (int k = 0; k < kPlanThreads / 32; ++k) {
    if (k < w) {
      bx += sx[k];
      bm += sm[k];
    }
    tx += sx[k];
    tm += sm[k];
  }
  x = bx + ix - x;  // exclusive
  m = bm + im - m;
  __syncthreads();
}

__global__ void __launch_bounds__(kPlanThreads) plan_count_kernel(CallArgs a, ClassCfg cc) {
  PlanCtx c = plan_ctx(a);
  const int p = blockIdx.x * kPlanThreads + threadIdx.x;
  int64_t xc = 0, mc = 0;
  if (p < c.P) {
    PairFacts f = pair_facts(c, p, cc);
    if (!f.valid) {
      set_status(c.hdr, 1 /* CF_ERR_INVALID_ARG */, p);
    } else {
      atomicAdd(&c.hdr->hist[f.cls][f.bucket], 1u);
      if (f.cls == kClassGlobal || f.cls == kClassCluster)  // both use a scratch slot
        atomicMax(reinterpret_cast<unsigned long long*>(&c.hdr->slot_need),
                  (unsigned long long)global_slot_bytes(f.na, f.nb));
      atomicMax(reinterpret_cast<unsigned long long*>(&c.hdr->bwd_slot_need),
                (unsigned long long)bwd_slot_bytes(f.na, f.nb, f.ea, f.eb, a.K, c.A.F_pad));
      // the adjoint's per-team slots of pairs not resident in one CTA: the
      // full-matrix layout of the cluster tier, or the global tier's own
      if (cc.bwd && (f.cls == kClassGlobal || f.cls == kClassCluster))
        atomicMax(reinterpret_cast<unsigned long long*>(&c.hdr->bwd_big_need),
                  (unsigned long long)(f.cls == kClassCluster ? bwd_res_slot_bytes(f.n_row, f.ld, a.K)
                                                              : bwd_slot_bytes(f.na, f.nb, f.ea, f.eb, a.K,
                                                                               c.A.F_pad)));
      xc = (int64_t)f.na * f.nb;
      mc = f.na;
    }
  }
  int64_t tx, tm;
  block_scan2(xc, mc, tx, tm);
  if (threadIdx.x == 0) {
    c.bsum[blockIdx.x] = tx;
    c.bsum[c.nblk + blockIdx.x] = tm;
  }
}

__global__ void __launch_bounds__(kPlanThreads) plan_scan_kernel(CallArgs a, int ranked) {
  PlanCtx c = plan_ctx(a);
  if (threadIdx.x == 0) {
    // queue order: class by class; within a class, costliest bucket first
    uint32_t pos = 0;
    for (int cls = 0; cls < kNumClasses; ++cls) {
      uint32_t start = pos;
      for (int b = kBuckets - 1; b >= 0; --b) {
        c.hdr->cursor[cls][b] = pos;
        pos += c.hdr->hist[cls][b];
      }
      c.hdr->n_class[cls] = pos - start;
    }
  }
  // exclusive scan of the per-block offset sums (chunked over the threads)
  const int per = ceil_div(c.nblk, kPlanThreads);
  const int b0 = threadIdx.x * per, b1 = min(c.nblk, b0 + per);
  int64_t sx = 0, sm = 0;
  for (int b = b0; b < b1; ++b) {
    sx += c.bsum[b];
    sm += c.bsum[c.nblk + b];
  }
  int64_t tx, tm;
  block_scan2(sx, sm, tx, tm);
  for (int b = b0; b < b1; ++b) {
    int64_t vx = c.bsum[b], vm = c.bsum[c.nblk + b];
    c.bsum[b] = sx;
    c.bsum[c.nblk + b] = sm;
    sx += vx;
    sm += vm;
  }
  if (threadIdx.x == 0) {
    c.hdr->x_total = tx;
    c.hdr->m_total = tm;
    c.x_off[c.P] = tx;
    c.m_off[c.P] = tm;
    // matching policy 3: the deferred-steps area at the end of the
    // workspace, if it fits beside one scratch slot (when any pair needs one)
    if (ranked == 3) {
      const WsLayout L = ws_layout(c.P);
      const size_t need = defer_bytes(c.P, tx);
      const size_t avail = a.ws_bytes > L.scratch ? a.ws_bytes - L.scratch : 0;
      const size_t slot =
          c.hdr->n_class[kClassGlobal] + c.hdr->n_class[kClassCluster] > 0 ? (size_t)c.hdr->slot_need : 0;
      if (need + slot <= avail) {
        c.hdr->defer = 1;
        c.hdr->defer_off = (a.ws_bytes - need + kAlign - 1) / kAlign * kAlign;
      }
    }
  }
}

__global__ void __launch_bounds__(kPlanThreads) plan_scatter_kernel(CallArgs a, ClassCfg cc) {
  PlanCtx c = plan_ctx(a);
  const int p = blockIdx.x * kPlanThreads + threadIdx.x;
  int64_t xc = 0, mc = 0;
  if (p < c.P) {
    PairFacts f = pair_facts(c, p, cc);
    if (f.valid) {
      uint32_t pos = atomicAdd(&c.hdr->cursor[f.cls][f.bucket], 1u);
      c.queue[pos] = (uint32_t)p;
      xc = (int64_t)f.na * f.nb;
      mc = f.na;
    }
  }
  int64_t tx, tm;
  block_scan2(xc, mc, tx, tm);
  if (p < c.P) {
    c.x_off[p] = c.bsum[blockIdx.x] + xc;
    c.m_off[p] = c.bsum[c.nblk + blockIdx.x] + mc;
  }
}

}  // namespace

cudaError_t launch_plan(const CallArgs& a, const ClassCfg& cc, cudaStream_t s) {
  WsLayout L = ws_layout(a.P);
  plan_count_kernel<<<L.plan_blocks, kPlanThreads, 0, s>>>(a, cc);
  plan_scan_kernel<<<1, kPlanThreads, 0, s>>>(a, cc.ranked);
  plan_scatter_kernel<<<L.plan_blocks, kPlanThreads, 0, s>>>(a, cc);
  return cudaGetLastError();
}

}  // namespace cfsim
