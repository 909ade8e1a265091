// Byte layouts shared by the host runtime and the kernels: the CSR batch pack,
// the workspace header, and the classification of a pair into an execution
// class (warp-, CTA- or global-memory-resident).  Plain C++ so that host-only
// translation units can include it.
#pragma once

#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define CF_HD __host__ __device__ __forceinline__
#else
#define CF_HD inline
#endif

namespace cfsim {

constexpr uint32_t kPackMagic = 0x4B504643u;  // "CFPK"
constexpr uint32_t kPackVersion = 2;
constexpr int kMaxBlocks = 32000;  // per CFG; matching state packs indices in int16
constexpr int kMaxF = 32;          // attributes per block
constexpr size_t kAlign = 256;

CF_HD size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
CF_HD int ceil_div(int a, int b) { return (a + b - 1) / b; }

// One adjacency entry: local index of the neighbour block and the edge weight.
struct CfAdj {
  int32_t nbr;
  float w;
};

// Header at byte 0 of a pack.  Every offset is in bytes from the pack base.
struct PackHeader {
  uint32_t magic, version;
  int32_t n_cfgs, F, F_pad, max_blocks;
  int32_t max_out_deg, max_in_deg;
  int64_t n_blocks, n_edges, n_user_edges, total_bytes;
  int64_t off_node;   // int32 [n_cfgs + 1]  first block of each CFG
  int64_t off_edge;   // int32 [n_cfgs + 1]  first distinct edge of each CFG
  int64_t off_uedge;  // int32 [n_cfgs + 1]  first user edge of each CFG
  int64_t off_out_ptr;  // int32 [n_blocks + 1] global index into out_adj per block
  int64_t off_in_ptr;   // int32 [n_blocks + 1] global index into in_adj per block
  int64_t off_out_adj;  // CfAdj [n_edges] sorted by (src, dst); position = distinct-edge id
  int64_t off_in_adj;   // CfAdj [n_edges] sorted by (dst, src)
  int64_t off_in_eid;   // int32 [n_edges] distinct-edge id of each in_adj entry
  int64_t off_u2c;      // int32 [n_user_edges] distinct-edge id of each user edge
  int64_t off_attr;     // float [n_blocks * F_pad]
  int64_t off_xdeg;     // uint8 [n_cfgs]: 1 if a block has more than two out- or in-neighbours
};

// Execution classes of a pair, in queue order: the global-memory tier, the
// five shared-memory group levels of the persistent kernel (whole CTA, half,
// quarter and eighth CTA, single warp), and the cluster tier (rows split over
// the CTAs of a thread-block cluster, iterate in distributed shared memory).
enum PairClass : int {
  kClassGlobal = 0,
  kClassCta = 1,
  kClassHalf = 2,
  kClassQuarter = 3,
  kClassEighth = 4,
  kClassWarp = 5,
  kClassCluster = 6,
  kNumClasses = 7,
  kClassSkip = 7
};
constexpr int kMaxCluster = 16;
constexpr int kBuckets = 64;  // cost buckets per class (two per octave)

// Shape of the batched forward kernel: threads per CTA and the shared-memory
// region (bytes) a pair may use at each group level.  The plan and the kernel
// classify pairs with the same values.
struct ClassCfg {
  int nt;       // threads per CTA (the CTA-level group)
  int z_cta;    // region of the CTA-level group
  int z_half;   // region of each of the two half groups (nt / 2 threads)
  int z_qtr;    // region of each of the four quarter groups (nt / 4 threads)
  int z_8th;    // region of each of the eight eighth groups (nt / 8 threads)
  int z_wrp;    // region of each warp
  int min_cls;  // smallest group level pairs may go to (kClassWarp: all levels)
  int ranked;   // matching of resident pairs: 0 ranked lists wherever their
                // state fits, 1 only in groups of at most a quarter CTA,
                // 2 never (rescans), 3 ranked lists wherever their state fits
                // with the sequential steps deferred to a second kernel
                // (one warp per pair) when the workspace has room
  int cluster;  // CTAs per cluster of the cluster tier (0: no cluster tier)
  int bwd;      // 1: size regions for the adjoint (bwd_resident_bytes), 0: the forward
};

// How a pair maps onto a group of G threads.  The "row" graph indexes the
// rows of the resident matrix, the "column" graph its columns; tr = 1 when
// the row graph is B (the matrix is then X^T).  Thread g < R * n_col owns
// column g % n_col and rows g / n_col + R * m, m < M.
struct Shape {
  int cls, tr, n_row, n_col, R, M, ld;
};

// Row stride of a resident pair's matrices: unpadded, so that the threads of a
// group, which take consecutive columns of consecutive rows, touch consecutive
// words in every sweep (an odd stride, which spreads a column over the banks
// for column rescans, put lanes two rows apart on the same bank: 1 % slower on
// the 19,900-pair workload).
CF_HD int pair_ld(int n_col) { return n_col; }

// Shared-memory bytes of a resident pair: (1 - alpha) Ehat and two iterates
// (n_row x ld floats each); per row of the row graph its first two out- and
// in-neighbours padded to two (two int4) and its full edge ranges (int4);
// the row graph's out- then in-edge entries and the column graph's out- then
// in-edge entries ({byte offset, w}, 8 bytes each); the column graph's out-
// and in-edge row pointers (int32, n_col + 1 each); the list of rows with
// more than two out- or in-neighbours (a count, then int16 pairs).
CF_HD size_t resident_bytes(int n_row, int ld, int e_row, int n_col, int e_col) {
  return align_up(12 * (size_t)n_row * ld, 16) + 48 * (size_t)n_row + 16 * (size_t)e_row + 16 * (size_t)e_col +
         align_up(8 * (size_t)(n_col + 1), 16) + align_up(8 + 4 * (size_t)n_row, 16);
}

// The adjoint keeps the same three matrices (the iterate being gathered, the
// next one or the adjoint being gathered, and a third), the same staged lists,
// and per edge of either graph its source ({row byte offset} or {column byte
// offset}, int32) and its gradient accumulator (float): 8 more bytes per edge.
CF_HD size_t bwd_resident_bytes(int n_row, int ld, int e_row, int n_col, int e_col) {
  return resident_bytes(n_row, ld, e_row, n_col, e_col) + align_up(8 * (size_t)(e_row + e_col), 16);
}

CF_HD size_t pair_bytes(int n_row, int ld, int e_row, int n_col, int e_col, int bwd) {
  return bwd ? bwd_resident_bytes(n_row, ld, e_row, n_col, e_col) : resident_bytes(n_row, ld, e_row, n_col, e_col);
}

CF_HD bool fits(int n_row, int n_col, int e_row, int e_col, int G, size_t region, int* R, int* M, int bwd = 0) {
  if (n_col > G) return false;
  *R = G / n_col;
  *M = ceil_div(n_row, *R);
  return pair_bytes(n_row, pair_ld(n_col), e_row, n_col, e_col, bwd) <= region;
}

CF_HD int group_size(int cls, const ClassCfg& c) {
  return cls == kClassWarp      ? 32
         : cls == kClassEighth  ? c.nt / 8
         : cls == kClassQuarter ? c.nt / 4
         : cls == kClassHalf    ? c.nt / 2
                                : c.nt;
}

CF_HD size_t group_region(int cls, const ClassCfg& c) {
  return (size_t)(cls == kClassWarp      ? c.z_wrp
                  : cls == kClassEighth  ? c.z_8th
                  : cls == kClassQuarter ? c.z_qtr
                  : cls == kClassHalf    ? c.z_half
                                         : c.z_cta);
}

// Orientation of a pair that fits both ways: the column graph's lists live in
// each thread's registers (its first two neighbours) and a column with more
// than two neighbours makes its lane run extra work while the rest of its warp
// waits, whereas a row's further neighbours are handled by whole warps.  So a
// CFG with such blocks (xa / xb) goes to the row side when the other has none;
// otherwise fewest rows per thread (ties: untransposed).
CF_HD bool prefer_tr(int M0, int M1, int xa, int xb) {
  if ((xa != 0) != (xb != 0)) return xb != 0;  // B has the busy blocks: make B the row graph
  return M1 < M0;
}

// Smallest group level (not below c.min_cls) whose region holds the pair,
// oriented by prefer_tr.  xa / xb: whether CFG A / B has a block with more
// than two out- or in-neighbours.
CF_HD Shape classify(int na, int nb, int ea, int eb, const ClassCfg& c, int xa = 0, int xb = 0) {
  Shape s{};
  for (int cls = c.min_cls; cls >= kClassCta; --cls) {
    const int G = group_size(cls, c);
    const size_t Z = group_region(cls, c);
    int R0 = 0, M0 = 0, R1 = 0, M1 = 0;
    const bool f0 = fits(na, nb, ea, eb, G, Z, &R0, &M0, c.bwd);
    const bool f1 = fits(nb, na, eb, ea, G, Z, &R1, &M1, c.bwd);
    if (f0 || f1) {
      const bool tr = !f0 || (f1 && prefer_tr(M0, M1, xa, xb));
      s.cls = cls;
      s.tr = tr ? 1 : 0;
      s.n_row = tr ? nb : na;
      s.n_col = tr ? na : nb;
      s.R = tr ? R1 : R0;
      s.M = tr ? M1 : M0;
      s.ld = pair_ld(s.n_col);
      return s;
    }
  }
  if (c.cluster >= 2) {
    // rows in c.cluster slabs, one per CTA; each CTA holds its slab of the
    // three matrices, its slab's row lists and the whole column graph
    int M0 = 0, M1 = 0;
    const int s0 = ceil_div(na, c.cluster), s1 = ceil_div(nb, c.cluster);
    const bool f0 = nb <= c.nt && pair_bytes(s0, pair_ld(nb), ea, nb, eb, c.bwd) <= (size_t)c.z_cta;
    const bool f1 = na <= c.nt && pair_bytes(s1, pair_ld(na), eb, na, ea, c.bwd) <= (size_t)c.z_cta;
    if (f0) M0 = ceil_div(s0, c.nt / nb);
    if (f1) M1 = ceil_div(s1, c.nt / na);
    if (f0 || f1) {
      const bool tr = !f0 || (f1 && prefer_tr(M0, M1, xa, xb));
      s.cls = kClassCluster;
      s.tr = tr ? 1 : 0;
      s.n_row = tr ? nb : na;
      s.n_col = tr ? na : nb;
      s.R = c.nt / s.n_col;
      s.M = tr ? M1 : M0;
      s.ld = pair_ld(s.n_col);
      return s;
    }
  }
  s.cls = kClassGlobal;
  s.tr = 0;
  s.n_row = na;
  s.n_col = nb;
  s.R = 0;
  s.M = 0;
  s.ld = nb;
  return s;
}

// Scratch a global-class pair needs: three n_a x n_b float matrices (two
// iterates and Ehat), row/column norms and the int32 matching state.
CF_HD size_t global_slot_bytes(int na, int nb) {
  size_t e = (size_t)na * nb;
  // Ehat, two iterates, norms, matching state, and 64 busy-column sums per row
  return align_up(4 * (3 * e + 2 * (size_t)(na + nb) + 2 * (size_t)na + nb + 64 + 64 * (size_t)na), kAlign);
}

// Adjoint checkpoints: X_k is kept for k = 0, S, 2S, ... with S = ceil(sqrt(K)),
// and each segment of S steps is recomputed from its checkpoint.
CF_HD int bwd_segment(int K) {
  int s = 1;
  while (s * s < K) ++s;
  return s;
}

// Adjoint scratch of one pair (n_a x n_b matrices, row-major, stride n_b):
// E, Ehat, Ehat-bar, X-bar, Z-bar, the checkpoints and one segment of
// iterates; the squared-norm history; attribute norms; both graphs' edge lists
// (source, target, weight) and their gradient accumulators; per-row
// projections for the omega gradient.
CF_HD size_t bwd_slot_bytes(int na, int nb, int ea, int eb, int K, int Fp) {
  const size_t E = (size_t)na * nb;
  const int S = bwd_segment(K);
  const int nck = K / S + 1;
  const size_t floats = E * (5 + (size_t)nck + (size_t)S + 1) + (size_t)(K + 2) + 2 * (size_t)(na + nb) +
                        4 * (size_t)(ea + eb) + (size_t)na * Fp + 64;
  return align_up(4 * floats, kAlign);
}

// Matrices of n_row x ld floats in the global (L2-resident) slot of a pair
// whose adjoint runs resident in shared memory: the checkpoints Y_0, Y_S, ...
// (K / S + 1), one segment of iterates (indices 1 .. S-1 of the segment; the
// last segment's Y_K lands at index K mod S), Ehat, the Ehat adjoint, and a
// stash of the X adjoint while a segment is recomputed.  Before them, the
// norms |Y_k|, k = 0 .. K, rounded up to 64 floats.
CF_HD int bwd_res_mats(int K) { return K / bwd_segment(K) + 1 + bwd_segment(K) + 3; }
CF_HD size_t bwd_res_norm_floats(int K) { return align_up((size_t)K + 2, 64); }
CF_HD size_t bwd_res_slot_bytes(int n_row, int ld, int K) {
  return align_up(4 * (bwd_res_norm_floats(K) + (size_t)n_row * ld * bwd_res_mats(K)), kAlign);
}

// Global-slot bytes per shared-memory byte of a group's region, in 1/256
// units: any pair a region of Z bytes holds has n_row ld <= Z / 12 (three
// matrices), so a slot of Z ratio / 256 bytes (less one alignment unit)
// holds its matrices and norms whenever Z >= z_min, the smallest region.
CF_HD uint64_t bwd_slot_ratio_q(int K, size_t z_min) {
  const uint64_t per_entry = 4 * (uint64_t)bwd_res_mats(K);  // bytes per entry
  const uint64_t fixed = 4 * bwd_res_norm_floats(K) + 4 * (uint64_t)bwd_res_mats(K) + 2 * kAlign;
  return (256 * per_entry + 11) / 12 + (256 * fixed + z_min - 1) / z_min + 1;
}
// Byte offset of the slot of a group whose region starts at byte ro of its
// CTA's shared memory, within that CTA's slot area.
CF_HD size_t bwd_slot_at(size_t ro, uint64_t ratio_q) { return align_up((size_t)(ro * ratio_q / 256), kAlign); }

// Cost bucket: two buckets per octave of the per-iteration work.
CF_HD int cost_bucket(int64_t cost) {
  int b = 0;
  uint64_t v = (uint64_t)(cost > 0 ? cost : 1);
  while (v >= 4 && b < kBuckets - 2) {  // b ~ 2 log2(cost) capped
    v >>= 1;
    b += 2;
  }
  if (v >= 3 && b < kBuckets - 1) b += 1;
  return b;
}

// Workspace header (first bytes of the workspace, zeroed at every call).
struct WsHeader {
  int32_t status;       // first device-side error (cf_status code), 0 = none
  int32_t status_info;  // pair index or other detail of that error
  uint32_t q_next[kNumClasses];
  uint32_t n_class[kNumClasses];
  uint64_t slot_need;      // bytes of scratch the largest global-class pair needs
  uint64_t bwd_slot_need;  // bytes of adjoint scratch the largest pair needs
  uint32_t q_bwd;          // adjoint work counter (one-CTA pairs)
  uint32_t q_bwd_big;      // adjoint work counter (pairs on clusters)
  uint64_t q_opt;          // optimal-matching work counter (64-bit: claimed by compare-and-swap)
  uint64_t bwd_big_need;   // adjoint scratch bytes of the largest cluster- or global-class pair
  uint32_t hist[kNumClasses][kBuckets];
  uint32_t cursor[kNumClasses][kBuckets];
  int64_t x_total, m_total;
  // deferred matching steps (matching policy 3): whether the plan found room
  // for the ranked lists, the byte offset of that area in the workspace, the
  // pairs deferred so far and the second kernel's work counter
  uint32_t defer, n_def, q_def, pad_;
  uint64_t defer_off;
};

// Bytes of the deferred-steps area for P pairs with x_total entries in all:
// every pair's ranked elements (int16) and ranked keys (uint32), the list of
// deferred pairs (uint32 each), and slack for aligning the area's start.
CF_HD size_t defer_bytes(int P, int64_t x_total) {
  return align_up(2 * (size_t)x_total, kAlign) + align_up(4 * (size_t)x_total, kAlign) +
         align_up(4 * (size_t)(P > 0 ? P : 1), kAlign) + kAlign;
}

// Byte offsets of the forward workspace sections for P pairs.
struct WsLayout {
  size_t hdr, queue, x_off, m_off, bsum, scratch, fixed_bytes;
  int plan_blocks;
};

constexpr int kPlanThreads = 256;

CF_HD WsLayout ws_layout(int P) {
  WsLayout L{};
  size_t o = 0;
  L.hdr = o;
  o = align_up(o + sizeof(WsHeader), kAlign);
  L.queue = o;
  o = align_up(o + 4 * (size_t)(P > 0 ? P : 1), kAlign);
  L.x_off = o;
  o = align_up(o + 8 * (size_t)(P + 1), kAlign);
  L.m_off = o;
  o = align_up(o + 8 * (size_t)(P + 1), kAlign);
  L.plan_blocks = ceil_div(P > 0 ? P : 1, kPlanThreads);
  L.bsum = o;
  o = align_up(o + 2 * 8 * (size_t)L.plan_blocks, kAlign);
  L.scratch = o;
  L.fixed_bytes = o;
  return L;
}

// Adjoint workspace: the forward's fixed part, one float per distinct edge of
// pack A and (unless both sides are the same pack) of pack B, then the slots.
struct BwdLayout {
  size_t grad_a, grad_b, slots;
};

CF_HD BwdLayout bwd_layout(int P, int64_t ne_a, int64_t ne_b, bool same) {
  BwdLayout B{};
  size_t o = ws_layout(P).fixed_bytes;
  B.grad_a = o;
  o = align_up(o + 4 * (size_t)(ne_a > 0 ? ne_a : 1), kAlign);
  B.grad_b = same ? B.grad_a : o;
  if (!same) o = align_up(o + 4 * (size_t)(ne_b > 0 ? ne_b : 1), kAlign);
  B.slots = o;
  return B;
}

}  // namespace cfsim
