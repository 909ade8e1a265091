// a2-a7: the batched similarity forward, greedy matching and graph score.
//
// One persistent kernel, one 1024-thread CTA per SM, drains six cost-ordered
// queues (filled by plan.cu), largest work first:
//   global class:  pairs too large for shared memory; the whole CTA iterates X
//                  in a scratch slot of the workspace (L2-resident),
//   CTA class:     the whole CTA keeps the pair in its 220 KB of shared memory,
//   half class:    two 512-thread groups (named barriers 5-6) each keep a pair
//                  in their half of the shared memory,
//   quarter class: four 256-thread groups (named barriers 1-4) each keep a
//                  pair in their quarter of the shared memory,
//   eighth class:  eight 128-thread groups (named barriers 7-14) each keep a
//                  pair in their eighth of the shared memory,
//   warp class:    every warp keeps a small pair in its own 1/32 slice.
// A group that finds its queue empty goes straight on to the next level's
// pairs in its own part of the shared memory, so the tail of one class
// overlaps the next.
//
// Iteration (Table 1 "Iso" row, IsoRank-style, renormalised every step):
//   Y_{k+1} = alpha/2 (W_A X_k W_B^T + W_A^T X_k W_B) + (1 - alpha) Ehat,
//   X_{k+1} = Y_{k+1} / |Y_{k+1}|_F.
// The kernel stores Y (unnormalised) and carries s_k = 1/|Y_k|: because the
// propagation is linear, Z(X_k) = s_k Z(Y_k), so the norm is only needed after
// the gathers, and each iteration has a single group barrier (inside the
// fused Frobenius-norm reduction) with Y double-buffered.
//
// Thread mapping of a resident pair (Shape in layout.h): thread g owns column
// j = g % n_col and rows r0 + R m.  The column graph's adjacency lists of j
// (first two entries, the common CFG degree) live in registers for the whole
// pair.  The row graph's lists are staged once per pair in shared memory as
// per-row edge ranges and {u * ld, w} entries, so a gather is two dependent
// shared loads and the lanes sharing a row read the same words.
#include <mutex>
#include <type_traits>

#include "device_common.cuh"
#include "device_state.h"
#include "iterate.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

struct Ctx {
  PackView A, B;
  const int32_t* pairs;
  float alpha;
  int K, norm_mode;
  float* X;
  float* scores;
  int32_t* match;
  const int64_t* x_off;
  const int64_t* m_off;
  const uint32_t* queue;
  WsHeader* hdr;
  unsigned char* scratch;
  size_t scratch_bytes;
  const float* om;    // omega, shared-memory copy
  const float* sqom;  // sqrt(omega), shared-memory copy
  int F, Fp;
  int ranked;  // matching policy (ClassCfg::ranked)
  // matching policy 3 with room in the workspace: where the ranked lists of
  // each pair go (at x_off[p]) and the list of deferred pairs
  int16_t* def_rk;
  uint32_t* def_rkey;
  uint32_t* def_list;
};

// One pair, oriented: the row graph indexes rows of the resident matrix.
struct Geo {
  Shape s;
  int p, na, nb;
  const int32_t* r_optr;
  const int32_t* r_iptr;
  const CfAdj* r_oadj;
  const CfAdj* r_iadj;
  const float* r_attr;
  const int32_t* c_optr;
  const int32_t* c_iptr;
  const CfAdj* c_oadj;
  const CfAdj* c_iadj;
  const float* c_attr;
};

__device__ __forceinline__ Geo make_geo(const Ctx& cx, int p, const ClassCfg& cc) {
  Geo g;
  g.p = p;
  const int pa = __ldg(cx.pairs + 2 * p), pb = __ldg(cx.pairs + 2 * p + 1);
  const int ba = __ldg(cx.A.node_off + pa), bb = __ldg(cx.B.node_off + pb);
  g.na = __ldg(cx.A.node_off + pa + 1) - ba;
  g.nb = __ldg(cx.B.node_off + pb + 1) - bb;
  const int ea = __ldg(cx.A.edge_off + pa + 1) - __ldg(cx.A.edge_off + pa);
  const int eb = __ldg(cx.B.edge_off + pb + 1) - __ldg(cx.B.edge_off + pb);
  g.s = classify(g.na, g.nb, ea, eb, cc, __ldg(cx.A.xdeg + pa), __ldg(cx.B.xdeg + pb));
  const PackView& R = g.s.tr ? cx.B : cx.A;
  const PackView& C = g.s.tr ? cx.A : cx.B;
  const int rb = g.s.tr ? bb : ba, cbse = g.s.tr ? ba : bb;
  g.r_optr = R.out_ptr + rb;
  g.r_iptr = R.in_ptr + rb;
  g.r_oadj = R.out_adj;
  g.r_iadj = R.in_adj;
  g.r_attr = R.attr + (size_t)rb * cx.Fp;
  g.c_optr = C.out_ptr + cbse;
  g.c_iptr = C.in_ptr + cbse;
  g.c_oadj = C.out_adj;
  g.c_iadj = C.in_adj;
  g.c_attr = C.attr + (size_t)cbse * cx.Fp;
  return g;
}

// Same sum with both graphs' lists read from memory (global-class pairs).
__device__ __forceinline__ float gather_g(const float* Y, int ld, const Geo& g, int i, int j) {
  float s = 0.f;
  const int c0 = __ldg(g.c_optr + j), c1 = __ldg(g.c_optr + j + 1);
  for (int e = __ldg(g.r_optr + i), e1 = __ldg(g.r_optr + i + 1); e < e1; ++e) {
    const CfAdj a = ldg_adj(g.r_oadj + e);
    const float* row = Y + (size_t)a.nbr * ld;
    float t = 0.f;
    for (int f = c0; f < c1; ++f) {
      const CfAdj b = ldg_adj(g.c_oadj + f);
      t = fmaf(b.w, row[b.nbr], t);
    }
    s = fmaf(a.w, t, s);
  }
  const int d0 = __ldg(g.c_iptr + j), d1 = __ldg(g.c_iptr + j + 1);
  for (int e = __ldg(g.r_iptr + i), e1 = __ldg(g.r_iptr + i + 1); e < e1; ++e) {
    const CfAdj a = ldg_adj(g.r_iadj + e);
    const float* row = Y + (size_t)a.nbr * ld;
    float t = 0.f;
    for (int f = d0; f < d1; ++f) {
      const CfAdj b = ldg_adj(g.c_iadj + f);
      t = fmaf(b.w, row[b.nbr], t);
    }
    s = fmaf(a.w, t, s);
  }
  return s;
}

// a5-a6: greedy matching by rounds of locally dominant entries, and the score.
//
// Sequential greedy takes the largest remaining entry under the strict order
// (value desc, A index asc, B index asc).  An entry that is the largest of its
// row and of its column among the remaining rows/columns is taken by that
// greedy, so matching every such entry at once and repeating gives the same
// matching.  Within a row the order reduces to (value desc, column asc) and
// within a column to (value desc, row asc) in either orientation.
//
// State per row (rb) and column (cb): >= 0 best live partner, -2 not yet
// computed, -1 no candidate (only with NaN entries), <= -3 matched to -3 - v.
// A round has three barriers:
//   A  every live row whose best column died (or was never computed) rescans
//      the live columns (a warp per row), and every live row stamps its best
//      column with the round number in tg,
//   A' every stamped column whose best row died (or was never computed)
//      rescans the live rows.  A column no live row names cannot hold a
//      locally dominant entry this round, so its best is not needed; X_K is
//      close to rank one, so most rows name the same few columns and most
//      column rescans are skipped.  Liveness changes only in B, so these
//      scans agree, and a kept best stays right (bests only change when they
//      die).
//   B  every row whose best column names it back is matched; the round's
//      matches are counted by a group sum.  A row's entry is written only by
//      its own thread, a column's only by the thread of the row it names.
// Every round matches at least one pair for finite X (the largest live entry
// is locally dominant), so the loop is bounded by min(n_row, n_col) rounds; if
// the bound is reached first (NaN in X) the status word gets CF_ERR_NUMERIC.
// tg: n_col entries (round stamps, values up to min(n_row, n_col)).
// Returns the score on every thread; writes match[n_a] if given.
template <class IdxT, class Grp>
__device__ __forceinline__ float greedy(const Grp& grp, const float* X, int ld, int n_row, int n_col, int tr,
                                        IdxT* rb, IdxT* cb, IdxT* tg, int32_t* mo, WsHeader* hdr, int pidx) {
  const int t = grp.rank, G = grp.size, lane = t & 31, w = grp.warp(), NW = grp.nwarps();
  for (int r = t; r < n_row; r += G) rb[r] = (IdxT)-2;
  for (int c = t; c < n_col; c += G) {
    cb[c] = (IdxT)-2;
    tg[c] = (IdxT)0;
  }
  grp.sync();
  const int need = min(n_row, n_col);
  int matched = 0, par = 0;
  for (int round = 0; matched < need && round < need; ++round) {
    const IdxT stamp = (IdxT)(round + 1);
    for (int r = w; r < n_row; r += NW) {
      int v = rb[r];
      if (v <= -3) continue;  // matched
      if (v == -2 || (v >= 0 && cb[v] <= (IdxT)-3)) {
        float bv = -CUDART_INF_F;
        int bi = 0x7fffffff;
        const float* xr = X + (size_t)r * ld;
        for (int c = lane; c < n_col; c += 32)
          if (cb[c] > (IdxT)-3) {
            const float x = xr[c];
            if (x > bv) {
              bv = x;
              bi = c;
            }
          }
        warp_argmax(bv, bi);
        v = bi == 0x7fffffff ? -1 : bi;
        if (lane == 0) rb[r] = (IdxT)v;
      }
      if (lane == 0 && v >= 0) tg[v] = stamp;
    }
    grp.sync();
    for (int c = w; c < n_col; c += NW) {
      if (tg[c] != stamp) continue;  // no live row names it
      const int v = cb[c];
      if (!(v == -2 || (v >= 0 && rb[v] <= (IdxT)-3))) continue;
      float bv = -CUDART_INF_F;
      int bi = 0x7fffffff;
      for (int r = lane; r < n_row; r += 32)
        if (rb[r] > (IdxT)-3) {
          const float x = X[(size_t)r * ld + c];
          if (x > bv) {
            bv = x;
            bi = r;
          }
        }
      warp_argmax(bv, bi);
      if (lane == 0) cb[c] = bi == 0x7fffffff ? (IdxT)-1 : (IdxT)bi;
    }
    grp.sync();
    int nn = 0;
    for (int r = t; r < n_row; r += G) {
      const int c = rb[r];
      if (c >= 0 && cb[c] == r) {
        rb[r] = (IdxT)(-3 - c);
        cb[c] = (IdxT)(-3 - r);
        ++nn;
      }
    }
    matched += grp.sum_i(nn, par);
    par ^= 1;
  }
  if (matched < need && t == 0 && hdr) set_status(hdr, 6 /* CF_ERR_NUMERIC */, pidx);
  float sc = 0.f;
  if (!tr) {
    for (int r = t; r < n_row; r += G) {
      const int v = rb[r];
      const int c = v <= -3 ? -3 - v : -1;
      if (c >= 0) sc += X[(size_t)r * ld + c];
      if (mo) mo[r] = c;
    }
  } else {
    for (int c = t; c < n_col; c += G) {
      const int v = cb[c];
      const int r = v <= -3 ? -3 - v : -1;
      if (r >= 0) sc += X[(size_t)r * ld + c];
      if (mo) mo[c] = r;
    }
  }
  return grp.sum(sc, 0);
}

// a5-a6 for shared-memory-resident pairs: the same rounds of locally
// dominant entries as greedy(), but every row's columns and every column's
// rows are ranked once (value desc, index asc; the within-row and
// within-column parts of the greedy order), so finding a row's best live
// column is a cursor advance past dead entries of its ranked list instead of
// a rescan.  One thread per row / column, two group barriers per round.
// rs: ranked columns of each row [n_row][n_col], cs: ranked rows of each
// column [n_col][n_row] (int16); cursors, bests and dead flags per row and
// column.  An entry written by no rank (NaN in X) is skipped as dead.
__device__ __forceinline__ float greedy_ranked(const Group& grp, const float* X, int ld, int n_row, int n_col,
                                               int tr, int16_t* rs, int16_t* cs, unsigned char* st, int32_t* mo,
                                               WsHeader* hdr, int pidx) {
  const int t = grp.rank, G = grp.size;
  int16_t* rcur = reinterpret_cast<int16_t*>(st);
  int16_t* ccur = rcur + n_row;
  int16_t* rbest = ccur + n_col;
  int16_t* cbest = rbest + n_row;
  unsigned char* rdead = reinterpret_cast<unsigned char*>(cbest + n_col);
  unsigned char* cdead = rdead + n_row;
  const int E = n_row * n_col;
  for (int idx = t; idx < E; idx += G) {
    const int r = idx / n_col, c = idx - r * n_col;
    const float* xr = X + (size_t)r * ld;
    const float x = xr[c];
    int kr = 0;
    for (int c2 = 0; c2 < n_col; ++c2) {
      const float y = xr[c2];
      kr += (y > x) | ((y == x) & (c2 < c));
    }
    int kc = 0;
    for (int r2 = 0; r2 < n_row; ++r2) {
      const float y = X[(size_t)r2 * ld + c];
      kc += (y > x) | ((y == x) & (r2 < r));
    }
    if (kr < n_col) rs[r * n_col + kr] = (int16_t)c;
    if (kc < n_row) cs[c * n_row + kc] = (int16_t)r;
  }
  for (int r = t; r < n_row; r += G) {
    rcur[r] = 0;
    rdead[r] = 0;
  }
  for (int c = t; c < n_col; c += G) {
    ccur[c] = 0;
    cdead[c] = 0;
  }
  grp.sync();
  const int need = min(n_row, n_col);
  int matched = 0, par = 0;
  for (int round = 0; matched < need && round < need; ++round) {
    for (int r = t; r < n_row; r += G) {
      if (rdead[r]) continue;
      int k = rcur[r], c = -1;
      for (; k < n_col; ++k) {
        const int v = rs[r * n_col + k];
        if ((unsigned)v < (unsigned)n_col && !cdead[v]) {
          c = v;
          break;
        }
      }
      rcur[r] = (int16_t)k;
      rbest[r] = (int16_t)c;
    }
    for (int c = t; c < n_col; c += G) {
      if (cdead[c]) continue;
      int k = ccur[c], r = -1;
      for (; k < n_row; ++k) {
        const int v = cs[c * n_row + k];
        if ((unsigned)v < (unsigned)n_row && !rdead[v]) {
          r = v;
          break;
        }
      }
      ccur[c] = (int16_t)k;
      cbest[c] = (int16_t)r;
    }
    grp.sync();
    int nn = 0;
    for (int r = t; r < n_row; r += G) {
      if (rdead[r]) continue;
      const int c = rbest[r];
      if (c >= 0 && cbest[c] == r) {
        rdead[r] = 1;
        cdead[c] = 1;
        ++nn;
      }
    }
    matched += grp.sum_i(nn, par);
    par ^= 1;
  }
  if (matched < need && t == 0 && hdr) set_status(hdr, 6 /* CF_ERR_NUMERIC */, pidx);
  float sc = 0.f;
  for (int r = t; r < n_row; r += G)
    if (rdead[r]) sc += X[(size_t)r * ld + rbest[r]];
  if (mo) {
    if (!tr)
      for (int r = t; r < n_row; r += G) mo[r] = rdead[r] ? rbest[r] : -1;
    else
      for (int c = t; c < n_col; c += G) mo[c] = cdead[c] ? cbest[c] : -1;
  }
  return grp.sum(sc, 0);
}

// a5-a6 as the sequential greedy itself, on one warp.
//
// Every entry gets an order key okey(x): unsigned comparison of keys is the
// float order, NaN lowest (after -inf, where the greedy order visits it) and
// -0 equal to +0; keys are >= 1 so that 0 marks a finished list.  Lists run
// along the shorter side: a list is a row when n_col <= n_row, else a column,
// and it ranks its len = min(n_row, n_col) elements by (key desc, index asc),
// which is the greedy order (value desc, A index asc, B index asc) restricted
// to the list in either orientation.  The whole group counts the ranks, len
// comparisons per entry (the rounds of greedy_ranked rank both sides).  Then
// one warp takes the greedy's entries in turn: the head of every live list is
// its best live element, and the best head under the greedy order (key desc,
// then (A, B) index asc) is the largest live entry, the one sequential greedy
// takes next.  Its list and element die, and the lists whose head was that
// element advance past dead elements.  Exactly len steps, each a warp-wide
// max and min (redux.sync) over the heads held in registers (R per lane), with
// no group barrier.
// Shared memory: key n_row x ld (the free iterate); the ranked elements rk
// (int16, nl x len) and then the dead flags (len bytes) over X_K, which the
// keys replace; the ranked keys rkey (uint32, nl x len) over the Ehat buffer.
// Returns the score on the group's rank 0; writes match[n_A] (-1 for
// unmatched rows of A) if given.  A taken NaN entry sets CF_ERR_NUMERIC.
__device__ __forceinline__ uint32_t okey(float x) {
  if (x != x) return 1u;
  if (x == 0.f) x = 0.f;
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey_value(uint32_t k) {
  return k == 1u ? __int_as_float(0x7fffffff) : __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <int R>
__device__ __noinline__ float greedy_seq_steps(int lane, bool swap, int nl, int len, const int16_t* rk,
                                               const uint32_t* rkey, unsigned char* dead, int32_t* mo,
                                               WsHeader* hdr, int pidx) {
  // (A, B) index of element e of list l: (l, e), or (e, l) when swapped
  auto tie = [&](int l, int e) -> uint32_t {
    return swap ? ((uint32_t)e << 16) | (uint32_t)l : ((uint32_t)l << 16) | (uint32_t)e;
  };
  int cur[R], el[R];
  uint32_t hk[R], ht[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int l = lane + 32 * s;
    cur[s] = 0;
    el[s] = -1;
    hk[s] = 0u;
    ht[s] = 0xffffffffu;
    if (l < nl) {
      const int e = rk[l * len];
      el[s] = e;
      hk[s] = rkey[l * len];
      ht[s] = tie(l, e);
    }
  }
  float sc = 0.f;
  for (int step = 0; step < len; ++step) {
    uint32_t bk = 0u, bt = 0xffffffffu;
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (hk[s] > bk || (hk[s] == bk && ht[s] < bt)) {
        bk = hk[s];
        bt = ht[s];
      }
    const uint32_t mk = __reduce_max_sync(0xffffffffu, bk);
    const uint32_t mt = __reduce_min_sync(0xffffffffu, bk == mk ? bt : 0xffffffffu);
    if (mk == 0u) break;  // no live list (not reached: a live list remains while steps remain)
    const int hi = (int)(mt >> 16), lo = (int)(mt & 0xffffu);
    const int l = swap ? lo : hi, e = swap ? hi : lo;
    if (lane == 0) {
      dead[e] = 1;
      sc += okey_value(mk);
      if (mo) mo[hi] = lo;
      if (mk == 1u && hdr) set_status(hdr, 6 /* CF_ERR_NUMERIC */, pidx);
    }
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (lane + 32 * s == l) {  // the taken list
        el[s] = -1;
        hk[s] = 0u;
        ht[s] = 0xffffffffu;
      }
    if (step + 1 == len) break;  // every element is taken
    __syncwarp();                 // dead[e] is visible to the warp
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (el[s] == e) {  // its head died: the next live element of its list
        const int base = (lane + 32 * s) * len;
        int k = cur[s] + 1, v = -1;
        uint32_t kv = 0u;
        for (; k < len; ++k) {
          v = rk[base + k];
          kv = rkey[base + k];
          if (!dead[v]) break;
        }
        cur[s] = k;
        if (k < len) {
          el[s] = v;
          hk[s] = kv;
          ht[s] = tie(lane + 32 * s, v);
        } else {  // not reached: a live element remains while steps remain
          el[s] = -1;
          hk[s] = 0u;
          ht[s] = 0xffffffffu;
        }
      }
  }
  return sc;
}

__device__ __forceinline__ float greedy_seq(const Group& grp, float* X, int ld, int n_row, int n_col, int tr,
                                            uint32_t* key, uint32_t* rkey, int32_t* mo, WsHeader* hdr, int pidx,
                                            bool steps = true) {
  const int t = grp.rank, G = grp.size;
  const bool rows = n_col <= n_row;
  const int nl = rows ? n_row : n_col, len = rows ? n_col : n_row;
  const int E = n_row * n_col;
  for (int idx = t; idx < E; idx += G) {
    const int r = idx / n_col, c = idx - r * n_col;
    key[r * ld + c] = okey(X[r * ld + c]);
  }
  if (mo) {
    const int nA = tr ? n_col : n_row;
    for (int a = t; a < nA; a += G) mo[a] = -1;
  }
  grp.sync();
  // rank of element e in list l: elements with a larger key, or an equal key
  // and a smaller index (k >= 1, so k - 1 does not wrap)
  int16_t* rk = reinterpret_cast<int16_t*>(X);
  unsigned char* dead = reinterpret_cast<unsigned char*>(rk + nl * len);
  for (int idx = t; idx < E; idx += G) {
    const int r = idx / n_col, c = idx - r * n_col;
    const uint32_t k = key[r * ld + c];
    const int l = rows ? r : c, e = rows ? c : r;
    const uint32_t* kp = rows ? key + r * ld : key + c;
    const int st = rows ? 1 : ld;
    int cnt = 0;
#pragma unroll 4
    for (int e2 = 0; e2 < len; ++e2) cnt += kp[e2 * st] > k - (uint32_t)(e2 < e);
    rk[l * len + cnt] = (int16_t)e;
    rkey[l * len + cnt] = k;
  }
  for (int e = t; e < len; e += G) dead[e] = 0;
  grp.sync();
  float sc = 0.f;
  if (steps && t < 32) {
    const bool swap = rows == (tr != 0);
    const int Rn = (nl + 31) >> 5;
    if (Rn <= 1)
      sc = greedy_seq_steps<1>(t, swap, nl, len, rk, rkey, dead, mo, hdr, pidx);
    else if (Rn <= 2)
      sc = greedy_seq_steps<2>(t, swap, nl, len, rk, rkey, dead, mo, hdr, pidx);
    else if (Rn <= 4)
      sc = greedy_seq_steps<4>(t, swap, nl, len, rk, rkey, dead, mo, hdr, pidx);
    else
      sc = greedy_seq_steps<8>(t, swap, nl, len, rk, rkey, dead, mo, hdr, pidx);
  }
  return sc;
}
constexpr int kSeqMaxLists = 256;

// a5-a6 for a global-class pair on one CTA: the rounds of greedy(), with
// the row and column states in shared memory and both kinds of rescan
// reading contiguous memory.  A row rescan (a warp per row) reads the row of
// X_K; a column rescan (a warp per column) reads the row of X_K^T, written
// once into free scratch by 32 x 32 tiles through shared memory.  (With X_K
// in L2 or beyond, greedy()'s column scans -- one sector per lane per load --
// were the matching's cost.)  Each lane keeps four loads in flight.  The
// results are greedy()'s: the same rounds, the same per-line best under
// (value desc, index asc), NaN never taken.
// sm: rb (n_row), cb, tg (n_col each) as int16, then a 32 x 33 float tile
// per warp; XT: n_col x n_row floats of free scratch.
__device__ __forceinline__ void scan_line(const float* x, const int16_t* st, int n, int lane, float& bv, int& bi) {
  bv = -CUDART_INF_F;
  bi = 0x7fffffff;
  for (int c0 = lane; c0 < n; c0 += 128) {
    float v[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + 32 * u;
      ok[u] = c < n && st[c] > (int16_t)-3;
      v[u] = c < n ? x[c] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u] && v[u] > bv) {  // a lane's columns ascend: strict > keeps the smallest
        bv = v[u];
        bi = c0 + 32 * u;
      }
  }
  warp_argmax(bv, bi);
}

__device__ __noinline__ float greedy_g(const Group& grp, const float* X, int n_row, int n_col, float* XT,
                                       unsigned char* sm, int32_t* mo, WsHeader* hdr, int pidx) {
  const int t = grp.rank, G = grp.size, lane = t & 31, w = grp.warp(), NW = grp.nwarps();
  int16_t* rb = reinterpret_cast<int16_t*>(sm);
  int16_t* cb = rb + n_row;
  int16_t* tg = cb + n_col;
  float* tile = reinterpret_cast<float*>(align_up(reinterpret_cast<size_t>(tg + n_col), 16)) + w * 32 * 33;
  for (int r = t; r < n_row; r += G) rb[r] = (int16_t)-2;
  for (int c = t; c < n_col; c += G) {
    cb[c] = (int16_t)-2;
    tg[c] = 0;
  }
  // X^T by 32 x 32 tiles, a warp per tile
  const int tr = ceil_div(n_row, 32), tc = ceil_div(n_col, 32);
  for (int q = w; q < tr * tc; q += NW) {
    const int r0 = (q / tc) * 32, c0 = (q % tc) * 32;
    for (int k = 0; k < 32; ++k)
      if (r0 + k < n_row && c0 + lane < n_col) tile[k * 33 + lane] = X[(size_t)(r0 + k) * n_col + c0 + lane];
    __syncwarp();
    for (int k = 0; k < 32; ++k)
      if (c0 + k < n_col && r0 + lane < n_row) XT[(size_t)(c0 + k) * n_row + r0 + lane] = tile[lane * 33 + k];
    __syncwarp();
  }
  grp.sync();

  const int need = min(n_row, n_col);
  int matched = 0, par = 0;
  for (int round = 0; matched < need && round < need; ++round) {
    const int16_t stamp = (int16_t)(round + 1);
    for (int r = w; r < n_row; r += NW) {
      int v = rb[r];
      if (v <= -3) continue;  // matched
      if (v == -2 || (v >= 0 && cb[v] <= (int16_t)-3)) {
        float bv;
        int bi;
        scan_line(X + (size_t)r * n_col, cb, n_col, lane, bv, bi);
        v = bi == 0x7fffffff ? -1 : bi;
        if (lane == 0) rb[r] = (int16_t)v;
      }
      if (lane == 0 && v >= 0) tg[v] = stamp;
    }
    grp.sync();
    for (int c = w; c < n_col; c += NW) {
      if (tg[c] != stamp) continue;  // no live row names it
      const int v = cb[c];
      if (!(v == -2 || (v >= 0 && rb[v] <= (int16_t)-3))) continue;
      float bv;
      int bi;
      scan_line(XT + (size_t)c * n_row, rb, n_row, lane, bv, bi);
      if (lane == 0) cb[c] = bi == 0x7fffffff ? (int16_t)-1 : (int16_t)bi;
    }
    grp.sync();
    int nn = 0;
    for (int r = t; r < n_row; r += G) {
      const int c = rb[r];
      if (c >= 0 && cb[c] == r) {
        rb[r] = (int16_t)(-3 - c);
        cb[c] = (int16_t)(-3 - r);
        ++nn;
      }
    }
    matched += grp.sum_i(nn, par);
    par ^= 1;
  }
  if (matched < need && t == 0 && hdr) set_status(hdr, 6 /* CF_ERR_NUMERIC */, pidx);
  float sc = 0.f;
  for (int r = t; r < n_row; r += G) {
    const int v = rb[r];
    const int c = v <= -3 ? -3 - v : -1;
    if (c >= 0) sc += X[(size_t)r * n_col + c];
    if (mo) mo[r] = c;
  }
  return grp.sum(sc, 0);
}

// Write X_K (resident, possibly transposed, stride ld) to the caller's
// row-major n_a x n_b output, coalesced on the global side.
template <class Grp>
__device__ __forceinline__ void store_x(const Grp& grp, const Ctx& cx, const Geo& g, const float* Xs, int ld) {
  float* dst = cx.X + cx.x_off[g.p];
  const int tot = g.na * g.nb;
  for (int idx = grp.rank; idx < tot; idx += grp.size) {
    const int ia = idx / g.nb, jb = idx - ia * g.nb;
    const int r = g.s.tr ? jb : ia, c = g.s.tr ? ia : jb;
    dst[idx] = Xs[(size_t)r * ld + c];
  }
}

// A shared-memory-resident pair on a group.  Region layout (bytes):
//   [ (1-alpha) Ehat | Y0 | Y1 ]  3 x n_row*ld floats,
//   [ ra ]  int4 per row: first two out-neighbours {u ld 4, w}, padded; the
//           sign bit of the last word flags a row with > 2 out- or in-neighbours,
//   [ rq ]  int4 per row: first two in-neighbours, padded,
//   [ rr ]  int4 per row: its full out- and in-edge ranges into redge,
//   [ redge ] {u ld 4, w}: the row graph's out-edges, then in-edges,
//   [ cedge ] {v 4, w}: the column graph's out-edges, then in-edges,
//   [ cptr ]  the column graph's out- then in-row pointers into cedge,
//   [ busy ]  the number of rows with > 2 out- or in-neighbours, then for each
//             such row its index and its index mod R (int16).
// Before X_0 exists, Y0 and Y1 hold the unit attribute vectors of the rows
// and columns (stride sF floats) when they fit.  After the iterations the
// Ehat buffer holds the row matching state and the free iterate the column
// state (int16).
__device__ __forceinline__ void run_pair_s(const Ctx& cx, const Geo& g, const Group& grp, unsigned char* region,
                                           size_t zbytes) {
  const Shape& s = g.s;
  const int t = grp.rank;
  const int ld = s.ld;
  const int nn = s.n_row * ld;
  float* ehb = reinterpret_cast<float*>(region);
  float* buf0 = ehb + nn;
  float* buf1 = buf0 + nn;
  int4* ra = reinterpret_cast<int4*>(region + align_up(12 * (size_t)nn, 16));
  int4* rq = ra + s.n_row;
  int4* rr = rq + s.n_row;
  int2* redge = reinterpret_cast<int2*>(rr + s.n_row);

  // stage the row graph and the column graph's entries
  const int eo0 = __ldg(g.r_optr), ei0 = __ldg(g.r_iptr);
  const int e_row = __ldg(g.r_optr + s.n_row) - eo0;
  const int co0 = __ldg(g.c_optr), ci0 = __ldg(g.c_iptr);
  const int e_col = __ldg(g.c_optr + s.n_col) - co0;
  int2* cedge = redge + 2 * e_row;
  int* cptr = reinterpret_cast<int*>(cedge + 2 * e_col);
  int* nbusy = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(cptr) + align_up(8 * (size_t)(s.n_col + 1), 16));
  int16_t* brow = reinterpret_cast<int16_t*>(nbusy + 2);  // [n_busy][2]: row, row mod R
  // (uniform over the group: every thread skips the pair together)
  if (!bounds_ok(cx.hdr, (size_t)(reinterpret_cast<unsigned char*>(brow + 2 * s.n_row) - region) <= zbytes,
                 kSiteFwdRegion))
    return;
  for (int k = t; k < e_col; k += grp.size) {
    CfAdj a = ldg_adj(g.c_oadj + co0 + k), b = ldg_adj(g.c_iadj + ci0 + k);
    if (!bounds_ok(cx.hdr, (unsigned)a.nbr < (unsigned)s.n_col && (unsigned)b.nbr < (unsigned)s.n_col,
                   kSiteFwdColNbr))
      a.nbr = b.nbr = 0;
    cedge[k] = make_int2(4 * a.nbr, __float_as_int(a.w));
    cedge[e_col + k] = make_int2(4 * b.nbr, __float_as_int(b.w));
  }
  for (int k = t; k <= s.n_col; k += grp.size) {
    cptr[k] = __ldg(g.c_optr + k) - co0;
    cptr[s.n_col + 1 + k] = e_col + __ldg(g.c_iptr + k) - ci0;
  }
  for (int i = t; i < s.n_row; i += grp.size) {
    const int o0 = __ldg(g.r_optr + i) - eo0, o1 = __ldg(g.r_optr + i + 1) - eo0;
    const int q0 = __ldg(g.r_iptr + i) - ei0, q1 = __ldg(g.r_iptr + i + 1) - ei0;
    rr[i] = make_int4(o0, o1, e_row + q0, e_row + q1);
  }
  for (int k = t; k < e_row; k += grp.size) {
    CfAdj a = ldg_adj(g.r_oadj + eo0 + k), b = ldg_adj(g.r_iadj + ei0 + k);
    if (!bounds_ok(cx.hdr, (unsigned)a.nbr < (unsigned)s.n_row && (unsigned)b.nbr < (unsigned)s.n_row,
                   kSiteFwdRowNbr))
      a.nbr = b.nbr = 0;
    redge[k] = make_int2(4 * ld * a.nbr, __float_as_int(a.w));
    redge[e_row + k] = make_int2(4 * ld * b.nbr, __float_as_int(b.w));
  }
  // a2: unit attribute vectors of rows and columns in Y0/Y1 (free until X_0
  // is written), stride sF (an odd multiple of 4 floats: conflict-free float4
  // reads across lanes); pairs too small to hold them read the pack instead
  const int sF = cx.Fp | 4;
  const bool staged = 4 * (size_t)sF * (s.n_row + s.n_col) + 12 <= 8 * (size_t)nn;
  float* ahat = reinterpret_cast<float*>(align_up(reinterpret_cast<size_t>(buf0), 16));
  float* bhat = ahat + (size_t)s.n_row * sF;
  if (staged) {
    for (int k = t; k < s.n_row + s.n_col; k += grp.size) {
      if (k < s.n_row)
        unit_attr(g.r_attr + (size_t)k * cx.Fp, cx.sqom, cx.Fp, ahat + (size_t)k * sF);
      else
        unit_attr(g.c_attr + (size_t)(k - s.n_row) * cx.Fp, cx.sqom, cx.Fp, bhat + (size_t)(k - s.n_row) * sF);
    }
  } else {
    for (int i = t; i < s.n_row; i += grp.size) buf1[i] = attr_norm(g.r_attr + (size_t)i * cx.Fp, cx.om, cx.Fp);
  }
  const bool act = t < s.R * s.n_col;
  const int j = act ? t % s.n_col : 0;
  const int r0 = act ? t / s.n_col : 0;
  const int Mt = (act && s.n_row > r0) ? ceil_div(s.n_row - r0, s.R) : 0;
  const int step = s.R * ld;
  const int off0 = r0 * ld + j;
  grp.sync();  // staged lists and attribute vectors visible

  // a3: cosine attribute term E, its Frobenius norm, Ehat = X_0
  float ss = 0.f;
  if (staged) {
    const float4* bj = reinterpret_cast<const float4*>(bhat + (size_t)j * sF);
    for (int m = 0, i = r0, off = off0; m < Mt; ++m, i += s.R, off += step) {
      const float4* ai = reinterpret_cast<const float4*>(ahat + (size_t)i * sF);
      float e = 0.f;
      for (int q = 0; q < (cx.Fp >> 2); ++q) {
        const float4 u = ai[q], v = bj[q];
        e = fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, fmaf(u.w, v.w, e))));
      }
      ehb[off] = e;
      ss = fmaf(e, e, ss);
    }
  } else {
    const float* bc = g.c_attr + (size_t)j * cx.Fp;
    const float cj = attr_norm(bc, cx.om, cx.Fp);
    for (int m = 0, i = r0, off = off0; m < Mt; ++m, i += s.R, off += step) {
      const float dot = attr_dot(g.r_attr + (size_t)i * cx.Fp, bc, cx.om, cx.Fp);
      const float den = buf1[i] * cj;
      const float e = den > 0.f ? dot / den : 0.f;
      ehb[off] = e;
      ss = fmaf(e, e, ss);
    }
  }
  const float tot = grp.sum(ss, 0);  // also: every read of the attribute vectors is done
  const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  const float uni = 1.0f / sqrtf((float)s.n_row * (float)s.n_col);
  const float cb = 1.f - cx.alpha;
  for (int m = 0, off = off0; m < Mt; ++m, off += step) {
    const float eh = tot > 0.f ? ehb[off] * inv : uni;
    buf0[off] = eh;
    ehb[off] = cb * eh;
  }
  // The order in which each thread's rows are swept (warp 0 of the group,
  // into the free iterate, which the attribute vectors no longer occupy):
  // first the rows with at most one out- and one in-neighbour (most blocks
  // of a CFG), in index order, then the rest.  pos[i] = position of row i.
  // Also the rows with further neighbours, each with the thread slot
  // (position mod R) of the threads that sweep it.
  int16_t* pos = reinterpret_cast<int16_t*>(buf1);
  if (grp.warp() == 0) {
    const int lane = t & 31;
    int na = 0;
    for (int b = 0; b < s.n_row; b += 32) {
      const int i = b + lane;
      int4 e = i < s.n_row ? rr[i] : make_int4(0, 0, 0, 0);
      const bool x = i < s.n_row && e.y - e.x <= 1 && e.w - e.z <= 1;
      const unsigned msk = __ballot_sync(0xffffffffu, x);
      if (x) pos[i] = (int16_t)(na + __popc(msk & ((1u << lane) - 1u)));
      na += __popc(msk);
    }
    int nb = na, cnt = 0;
    for (int b = 0; b < s.n_row; b += 32) {
      const int i = b + lane;
      const int4 e = i < s.n_row ? rr[i] : make_int4(0, 0, 0, 0);
      const bool x = i < s.n_row && !(e.y - e.x <= 1 && e.w - e.z <= 1);
      const unsigned msk = __ballot_sync(0xffffffffu, x);
      const int p = nb + __popc(msk & ((1u << lane) - 1u));
      if (x) pos[i] = (int16_t)p;
      nb += __popc(msk);
      const bool bz = x && (e.y - e.x > 2 || e.w - e.z > 2);
      const unsigned bm = __ballot_sync(0xffffffffu, bz);
      if (bz) {
        const int q = cnt + __popc(bm & ((1u << lane) - 1u));
        brow[2 * q] = (int16_t)i;
        brow[2 * q + 1] = (int16_t)(p % s.R);
      }
      cnt += __popc(bm);
    }
    if (lane == 0) {
      nbusy[0] = cnt;
      nbusy[1] = na;
    }
  }
  grp.sync();  // staged column pointers, row order visible
  // the row records, by position p: ra[p] = {row i | first out-neighbour u
  // << 16, first in-neighbour u' | flags << 16, w_iu, w_u'i} (bit 16 of the
  // flags: further neighbours); rq[p] = the second out- and in-neighbours
  // {u ld 4, w, u' ld 4, w'} (rows past the first group only); missing
  // neighbours padded with {0, 0}
  for (int i = t; i < s.n_row; i += grp.size) {
    const int4 e = rr[i];
    const int p = pos[i];
    const int2 z2 = make_int2(0, 0);
    const int2 a0 = e.y > e.x ? redge[e.x] : z2, a1 = e.y > e.x + 1 ? redge[e.x + 1] : z2;
    const int2 b0 = e.w > e.z ? redge[e.z] : z2, b1 = e.w > e.z + 1 ? redge[e.z + 1] : z2;
    const unsigned rs = 4u * (unsigned)ld;
    const unsigned busy = (e.y - e.x > 2 || e.w - e.z > 2) ? 1u : 0u;
    ra[p] = make_int4((int)((unsigned)i | (((unsigned)a0.x / rs) << 16)), (int)(((unsigned)b0.x / rs) | (busy << 16)),
                      a0.y, b0.y);
    rq[p] = make_int4(a1.x, a1.y, b1.x, b1.y);
  }
  const int na_rows = nbusy[1];
  grp.sync();  // row records visible (pos is overwritten by the first iteration)
  const ColPad cl = load_col(cptr, cedge, s.n_col, j);

  // a4: K renormalised iterations, one barrier each.  The main sweep is the
  // straight-line 2 x 2 gather for every entry; then the further-neighbour
  // terms are added to the entries of busy rows (by each entry's owner) and
  // of busy columns (by the owner's whole warp), and the norm's partial sums
  // are updated by y_new^2 - y_old^2.
  const int nbr = *nbusy;
  // positions p = r0 + R m: the first m1 of them are rows of the first group
  const int m1 = (Mt > 0 && na_rows > r0) ? min(Mt, ceil_div(na_rows - r0, s.R)) : 0;
  const int ld4 = 4 * ld;
  float sk = 1.f;
  for (int k = 0; k < cx.K; ++k) {
    const char* cur = reinterpret_cast<const char*>((k & 1) ? buf1 : buf0);
    float* nxt = (k & 1) ? buf0 : buf1;
    const float ca = 0.5f * cx.alpha * sk;
    ss = 0.f;
    // rows with at most one out- and one in-neighbour: four loads
#pragma unroll 1
    for (int m = 0, p = r0; m < m1; ++m, p += s.R) {
      const int4 A = ra[p];
      const int i = A.x & 0xffff;
      const int uo = ((unsigned)A.x >> 16) * ld4, ui = (A.y & 0xffff) * ld4;
      const float a0 = lds_at(cur, uo, cl.vo0), a1 = lds_at(cur, uo, cl.vo1);
      const float b0 = lds_at(cur, ui, cl.vi0), b1 = lds_at(cur, ui, cl.vi1);
      const float so = __int_as_float(A.z) * fmaf(cl.wo1, a1, cl.wo0 * a0);
      const float si = __int_as_float(A.w) * fmaf(cl.wi1, b1, cl.wi0 * b0);
      const int off = i * ld + j;
      const float y = fmaf(ca, so + si, ehb[off]);
      nxt[off] = y;
      ss = fmaf(y, y, ss);
    }
    // the other rows: the straight-line 2 x 2 gather (eight loads)
#pragma unroll 1
    for (int m = m1, p = r0 + m1 * s.R; m < Mt; ++m, p += s.R) {
      const int4 A = ra[p], B2 = rq[p];
      const int i = A.x & 0xffff;
      const int4 Ao = make_int4(((unsigned)A.x >> 16) * ld4, A.z, B2.x, B2.y);
      const int4 Qi = make_int4((A.y & 0xffff) * ld4, A.w, B2.z, B2.w);
      const int off = i * ld + j;
      const float y = fmaf(ca, gather_fast(cur, Ao, Qi, cl), ehb[off]);
      nxt[off] = y;
      ss = fmaf(y, y, ss);
    }
    for (int q = 0; q < nbr; ++q) {
      if (Mt == 0 || brow[2 * q + 1] != r0) continue;  // a row of another thread
      const int i = brow[2 * q];
      const int off = i * ld + j;
      const float y0 = nxt[off];
      const float y = fmaf(ca, row_extra(cur, rr[i], redge, cl), y0);
      nxt[off] = y;
      ss += y * y - y0 * y0;
    }
    // a busy column's entries are shared out over the lanes of the warp
    // that holds it (its owner wrote them above; __syncwarp orders that)
    __syncwarp();
    for (unsigned bm = __ballot_sync(0xffffffffu, cl.flag && Mt > 0); bm; bm &= bm - 1) {
      const int bl = __ffs(bm) - 1;
      const int jb = __shfl_sync(0xffffffffu, j, bl), pb = __shfl_sync(0xffffffffu, r0, bl);
      const int mb = __shfl_sync(0xffffffffu, Mt, bl);
      for (int m = t & 31; m < mb; m += 32) {
        const int p = pb + m * s.R;
        const int4 A = ra[p], B2 = rq[p];
        const bool two = p >= na_rows;
        const int i = A.x & 0xffff;
        const int4 Ao = make_int4(((unsigned)A.x >> 16) * ld4, A.z, two ? B2.x : 0, two ? B2.y : 0);
        const int4 Qi = make_int4((A.y & 0xffff) * ld4, A.w, two ? B2.z : 0, two ? B2.w : 0);
        const int off = i * ld + jb;
        const float y0 = nxt[off];
        const float y = fmaf(ca, col_extra(cur, Ao, Qi, rr[i], redge, cedge, cptr, s.n_col, jb), y0);
        nxt[off] = y;
        ss += y * y - y0 * y0;
      }
    }
    const float yy = grp.sum(ss, (k + 1) & 1);
    sk = cx.norm_mode == 0 ? 1.0f / sqrtf(yy) : 1.f;
  }
  float* Xs = (cx.K & 1) ? buf1 : buf0;
  float* freeb = (cx.K & 1) ? buf0 : buf1;
  if (sk != 1.f)
    for (int m = 0, off = off0; m < Mt; ++m, off += step) Xs[off] *= sk;
  grp.sync();

  if (cx.X) store_x(grp, cx, g, Xs, ld);
  if (cx.scores || cx.match) {
    int32_t* mo = cx.match ? cx.match + cx.m_off[g.p] : nullptr;
    const bool ranked = cx.ranked == 0 || cx.ranked == 3 || (cx.ranked == 1 && 4 * grp.size <= (int)blockDim.x);
    if (cx.def_rk && max(s.n_row, s.n_col) <= kSeqMaxLists) {
      // ranked lists here, then copied out for the deferred steps
      greedy_seq(grp, Xs, ld, s.n_row, s.n_col, s.tr, reinterpret_cast<uint32_t*>(freeb),
                 reinterpret_cast<uint32_t*>(ehb), mo, cx.hdr, g.p, false);
      const int E = s.n_row * s.n_col;
      const int16_t* rk = reinterpret_cast<const int16_t*>(Xs);
      const uint32_t* rkey = reinterpret_cast<const uint32_t*>(ehb);
      int16_t* grk = cx.def_rk + cx.x_off[g.p];
      uint32_t* grkey = cx.def_rkey + cx.x_off[g.p];
      for (int idx = t; idx < E; idx += grp.size) {
        grk[idx] = rk[idx];
        grkey[idx] = rkey[idx];
      }
      if (t == 0) cx.def_list[atomicAdd(&cx.hdr->n_def, 1u)] = (uint32_t)g.p | ((uint32_t)s.tr << 31);
    } else if (ranked && max(s.n_row, s.n_col) <= kSeqMaxLists) {
      // keys in the free iterate, ranked elements over X_K, their keys over Ehat
      const float sc = greedy_seq(grp, Xs, ld, s.n_row, s.n_col, s.tr, reinterpret_cast<uint32_t*>(freeb),
                                  reinterpret_cast<uint32_t*>(ehb), mo, cx.hdr, g.p);
      if (cx.scores && t == 0) cx.scores[g.p] = sc;
    } else if (ranked && 5 * (size_t)(s.n_row + s.n_col) + 16 <= 4 * (size_t)nn) {  // room for the ranked lists' state
      const float sc = greedy_ranked(grp, Xs, ld, s.n_row, s.n_col, s.tr, reinterpret_cast<int16_t*>(ehb),
                                     reinterpret_cast<int16_t*>(ehb) + s.n_row * s.n_col,
                                     reinterpret_cast<unsigned char*>(freeb), mo, cx.hdr, g.p);
      if (cx.scores && t == 0) cx.scores[g.p] = sc;
    } else {
      const float sc = greedy<int16_t>(grp, Xs, ld, s.n_row, s.n_col, s.tr, reinterpret_cast<int16_t*>(ehb),
                                       reinterpret_cast<int16_t*>(freeb), reinterpret_cast<int16_t*>(freeb) + s.n_col,
                                       mo, cx.hdr, g.p);
      if (cx.scores && t == 0) cx.scores[g.p] = sc;
    }
  }
  grp.sync();
}

// Calls f(i, j, i * ld + j) for the entries t, t + G, t + 2G, ... of an
// n_row x n_col matrix in row-major order, stepping (i, j) without a division.
template <class Fn>
__device__ __forceinline__ void for_entries(int n_row, int n_col, int ld, int t, int G, Fn&& f) {
  const int di = G / n_col, dj = G % n_col;
  for (int i = t / n_col, j = t % n_col; i < n_row;) {
    f(i, j, (size_t)i * ld + j);
    i += di;
    j += dj;
    if (j >= n_col) {
      j -= n_col;
      ++i;
    }
  }
}

// The sweep of one iteration of a global-class pair whose graphs are staged
// in shared memory.  The entries are cut into strips -- one column j and a
// run of L consecutive rows -- and team thread t takes strips t, t + G, ...;
// the lanes of a warp hold consecutive columns of the same rows, so every
// gather and store is coalesced and the row records are broadcast.  Rows go
// U at a time: the records, the gathered values and (1 - alpha) Ehat of U
// rows are all loaded before any of them is used, which keeps U * 9 loads of
// each thread in flight (the iterates live in L2 or beyond, so a chain of
// dependent loads per entry would leave the sweep latency-bound).  Rows with
// further neighbours add those terms in place.  Columns with further
// neighbours (the STOP block, whose in-degree grows with every early return,
// and loop exits) are left out: their entries cost many times an ordinary
// one, so sweep_busy spreads them over the whole team instead of leaving
// them to the strips' owners.  Returns this thread's partial sum of y^2.
struct StripPlan {
  int L, total, rounds;
};

// S row segments of L rows, S chosen to minimise the entries of the most
// loaded thread, ceil(S n_col / G) ceil(n_row / S) (ties: fewer segments).
__device__ __forceinline__ StripPlan strip_plan(int n_row, int n_col, int G) {
  int bS = 1;
  long long best = -1;
  for (int S = 1; S <= 64 && S <= n_row; ++S) {
    const long long c = (long long)ceil_div(S * n_col, G) * ceil_div(n_row, S);
    if (best < 0 || c < best) {
      best = c;
      bS = S;
    }
  }
  const int L = ceil_div(n_row, bS);
  const int total = ceil_div(n_row, L) * n_col;
  return StripPlan{L, total, ceil_div(total, G)};
}

template <int U>
__device__ __forceinline__ float sweep_strips(const StripPlan& sp, int t, int G, int n_row, int n_col, int ld,
                                              const char* cur, float* nxt, const float* ehb, float ca,
                                              const int4* ra, const int4* rq, const int4* rr, const int2* redge,
                                              const int2* cedge, const int* cptr) {
  float ss = 0.f;
  for (int rd = 0; rd < sp.rounds; ++rd) {
    const int q = t + rd * G;
    const int j = q < sp.total ? q % n_col : 0;
    const ColPad cl = load_col(cptr, cedge, n_col, j);
    const bool act = q < sp.total && !cl.flag;
    const int i0 = act ? (q / n_col) * sp.L : 0;
    const int i1 = act ? min(n_row, i0 + sp.L) : 0;
    int i = i0;
    for (; i + U <= i1; i += U) {
      int4 A[U], Q[U];
      float z[U], e[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        A[u] = ra[i + u];
        Q[u] = rq[i + u];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        z[u] = gather_fast(cur, A[u], Q[u], cl);
        e[u] = ehb[(size_t)(i + u) * ld + j];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (A[u].w < 0) z[u] += row_extra(cur, rr[i + u], redge, cl);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float y = fmaf(ca, z[u], e[u]);
        nxt[(size_t)(i + u) * ld + j] = y;
        ss = fmaf(y, y, ss);
      }
    }
    for (; i < i1; ++i) {
      const int4 A = ra[i];
      float z = gather_fast(cur, A, rq[i], cl);
      if (A.w < 0) z += row_extra(cur, rr[i], redge, cl);
      const float y = fmaf(ca, z, ehb[(size_t)i * ld + j]);
      nxt[(size_t)i * ld + j] = y;
      ss = fmaf(y, y, ss);
    }
  }
  return ss;
}

// Terms of entry (i, j) from the further neighbours of column j, as
// col_extra, with each neighbour's loads issued four at a time.
__device__ __forceinline__ float col_extra_g(const char* Y, const int4 A, const int4 Q, const int4 rr,
                                             const int2* redge, const int2* cedge, const int* cptr, int n_col,
                                             int j) {
  float s = 0.f;
  const float a0 = fabsf(__int_as_float(A.y)), a1 = fabsf(__int_as_float(A.w));
  const float q0 = __int_as_float(Q.y), q1 = __int_as_float(Q.w);
  auto term = [&](int u0, int u1, float w0, float w1, int r0, int r1, int2 v) {
    float t = fmaf(w1, lds_at(Y, u1, v.x), w0 * lds_at(Y, u0, v.x));
    for (int k = r0 + 2; k < r1; ++k) {
      const int2 e = redge[k];
      t = fmaf(__int_as_float(e.y), lds_at(Y, e.x, v.x), t);
    }
    return __int_as_float(v.y) * t;
  };
  const int xo0 = cptr[j] + 2, xo1 = cptr[j + 1];
  const int xi0 = cptr[n_col + 1 + j] + 2, xi1 = cptr[n_col + 2 + j];
#pragma unroll 4
  for (int f = xo0; f < xo1; ++f) s += term(A.x, A.z, a0, a1, rr.x, rr.y, cedge[f]);
#pragma unroll 4
  for (int f = xi0; f < xi1; ++f) s += term(Q.x, Q.z, q0, q1, rr.z, rr.w, cedge[f]);
  return s;
}

// The entries of the columns with further neighbours (nbc of them, listed in
// bcol), every one computed in full -- first two neighbours, row extras,
// column extras -- by whichever team thread takes it: items t, t + G, ...
// of the nbc x n_row of them, consecutive items down a column.
__device__ __forceinline__ float sweep_busy(int nbc, const int16_t* bcol, int t, int G, int n_row, int n_col, int ld,
                                            const char* cur, float* nxt, const float* ehb, float ca,
                                            const int4* ra, const int4* rq, const int4* rr, const int2* redge,
                                            const int2* cedge, const int* cptr) {
  float ss = 0.f;
  const int items = nbc * n_row;
  for (int k = t; k < items; k += G) {
    const int b = k / n_row, i = k - b * n_row;
    const int j = bcol[b];
    const ColPad cl = load_col(cptr, cedge, n_col, j);
    const int4 A = ra[i], Q = rq[i], R4 = rr[i];
    const size_t off = (size_t)i * ld + j;
    const float e = ehb[off];
    float z = gather_fast(cur, A, Q, cl);
    if (A.w < 0) z += row_extra(cur, R4, redge, cl);
    z += col_extra_g(cur, A, Q, R4, redge, cedge, cptr, n_col, j);
    const float y = fmaf(ca, z, e);
    nxt[off] = y;
    ss = fmaf(y, y, ss);
  }
  return ss;
}

// Busy columns through per-row sums.  For a column j with further
// neighbours, entry (i, j) of the gathered sum is
//   sum_{i->u} w_iu S_j[u] + sum_{u->i} w_ui P_j[u],
//   S_j[u] = sum_{j->v} w_jv Y[u,v],  P_j[u] = sum_{v->j} w_vj Y[u,v],
// so the many neighbours of such a column (the STOP block collects an edge
// from every early return) are read once per row u, along that row, instead
// of once per entry with a stride of one row per lane.  bsum_rows writes the
// sums into T (n_row rows of kBusySlots floats: slot 2b = S, 2b + 1 = P of
// busy column b), a warp per row: the column lists are cut into sub-slots of
// at most eight entries (sub: cedge begin, count | slot << 8), a lane takes
// sub-slots lane and lane + 32 with their loads all in flight, and each
// slot's sub-slot partials are then added in table order (slots: first sub,
// count), so the sums do not depend on timing.  bsum_entries then computes
// every busy-column entry (nbc x n_row items, consecutive items along a
// row) from row i's neighbour lists and T.
constexpr int kBusySlots = 64;  // 2 x up to 32 busy columns
constexpr int kBusySubs = 64;   // sub-slots: two per lane

__device__ __forceinline__ void bsum_rows(int w, int NW, int lane, int n_row, int ld, const char* cur, int nsub,
                                          const int2* sub, int nslot, const int* slots, const int2* cedge,
                                          float* pw, float* T) {
  for (int u = w; u < n_row; u += NW) {
    const char* row = cur + (size_t)u * ld * 4;
    float part[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int si = lane + 32 * h;
      part[h] = 0.f;
      if (si < nsub) {
        const int2 e = sub[si];
        const int cnt = e.y & 0xff;
        float v[8], wt[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int2 ce = q < cnt ? cedge[e.x + q] : make_int2(0, 0);
          wt[q] = __int_as_float(ce.y);
          v[q] = lds_at(row, 0, ce.x);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) part[h] = fmaf(wt[q], v[q], part[h]);
      }
    }
    pw[lane] = part[0];
    pw[lane + 32] = part[1];
    __syncwarp();
    for (int sl = lane; sl < nslot; sl += 32) {
      const int f = slots[sl] & 0xffff, c = slots[sl] >> 16;
      float acc = 0.f;
      for (int q = 0; q < c; ++q) acc += pw[f + q];
      T[(size_t)u * kBusySlots + sl] = acc;
    }
    __syncwarp();
  }
}

__device__ __forceinline__ float bsum_entries(int nbc, const int16_t* bcol, int t, int G, int n_row, int ld,
                                              float* nxt, const float* ehb, float ca, const int4* ra, const int4* rq,
                                              const int4* rr, const int2* redge, const float* T) {
  float ss = 0.f;
  const unsigned rs = 4u * (unsigned)ld;  // byte stride of a row: row offsets A.x = 4 ld u
  const int items = nbc * n_row;
  for (int k = t; k < items; k += G) {
    const int i = k / nbc, b = k - i * nbc;
    const int j = bcol[b];
    const int4 A = ra[i], Q = rq[i], R4 = rr[i];
    const float* So = T + 2 * b;
    const float* Pi = T + 2 * b + 1;
    float z = fabsf(__int_as_float(A.y)) * So[((unsigned)A.x / rs) * kBusySlots] +
              fabsf(__int_as_float(A.w)) * So[((unsigned)A.z / rs) * kBusySlots] +
              __int_as_float(Q.y) * Pi[((unsigned)Q.x / rs) * kBusySlots] +
              __int_as_float(Q.w) * Pi[((unsigned)Q.z / rs) * kBusySlots];
    for (int q = R4.x + 2; q < R4.y; ++q) {
      const int2 e = redge[q];
      z = fmaf(__int_as_float(e.y), So[((unsigned)e.x / rs) * kBusySlots], z);
    }
    for (int q = R4.z + 2; q < R4.w; ++q) {
      const int2 e = redge[q];
      z = fmaf(__int_as_float(e.y), Pi[((unsigned)e.x / rs) * kBusySlots], z);
    }
    const size_t off = (size_t)i * ld + j;
    const float y = fmaf(ca, z, ehb[off]);
    nxt[off] = y;
    ss = fmaf(y, y, ss);
  }
  return ss;
}

// A global-class pair (too large for shared memory) on a team -- the whole
// CTA, or every CTA of a thread-block cluster: the iterates, (1-alpha) Ehat
// and the matching state live in a scratch slot of the workspace
// (L2-resident); each CTA stages the row and column graphs in its own shared
// memory exactly as for a resident pair, and the gather is the same
// straight-line code on global addresses.  The team sweeps the entries in
// row-major order (team rank t takes t, t + G, ...).  Slot: [ehb | buf0 |
// buf1] (n_row x n_col floats each), row norms, int32 matching state.
// loc: this CTA (for the staging); team: the threads sharing the pair.
template <bool kStaged, int U, class Grp>
__device__ __noinline__ void run_pair_g(const Ctx& cx, const Geo& g, const Group& loc, const Grp& grp, float* slot,
                                        unsigned char* region) {
  const int n_row = g.na, n_col = g.nb, ld = g.nb;  // global-class shapes are never transposed
  const size_t E = (size_t)n_row * n_col;
  float* ehb = slot;
  float* buf0 = ehb + E;
  float* buf1 = buf0 + E;
  float* rn = buf1 + E;
  int32_t* ms = reinterpret_cast<int32_t*>(rn + n_row + n_col);
  const int t = grp.rank, G = grp.size;
  int4* ra = reinterpret_cast<int4*>(region);
  int4* rq = ra + n_row;
  int4* rr = rq + n_row;
  int2* redge = reinterpret_cast<int2*>(rr + n_row);

  // stage both graphs (byte offsets of rows use the global row stride ld);
  // without staging (graphs too large for shared memory) only the row norms
  const int eo0 = __ldg(g.r_optr), ei0 = __ldg(g.r_iptr);
  const int e_row = __ldg(g.r_optr + n_row) - eo0;
  const int co0 = __ldg(g.c_optr), ci0 = __ldg(g.c_iptr);
  const int e_col = __ldg(g.c_optr + n_col) - co0;
  int2* cedge = redge + 2 * e_row;
  int* cptr = reinterpret_cast<int*>(cedge + 2 * e_col);
  for (int i = t; i < n_row + n_col; i += G)
    rn[i] = i < n_row ? attr_norm(g.r_attr + (size_t)i * cx.Fp, cx.om, cx.Fp)
                      : attr_norm(g.c_attr + (size_t)(i - n_row) * cx.Fp, cx.om, cx.Fp);
  const int lt = loc.rank, LG = loc.size;
  for (int i = lt; kStaged && i < n_row; i += LG) {
    const int o0 = __ldg(g.r_optr + i) - eo0, o1 = __ldg(g.r_optr + i + 1) - eo0;
    const int q0 = __ldg(g.r_iptr + i) - ei0, q1 = __ldg(g.r_iptr + i + 1) - ei0;
    const CfAdj z{0, 0.f};
    const CfAdj a0 = o1 > o0 ? ldg_adj(g.r_oadj + eo0 + o0) : z, a1 = o1 > o0 + 1 ? ldg_adj(g.r_oadj + eo0 + o0 + 1) : z;
    const CfAdj b0 = q1 > q0 ? ldg_adj(g.r_iadj + ei0 + q0) : z, b1 = q1 > q0 + 1 ? ldg_adj(g.r_iadj + ei0 + q0 + 1) : z;
    const int flag = (o1 - o0 > 2 || q1 - q0 > 2) ? (int)0x80000000 : 0;
    ra[i] = make_int4(4 * ld * a0.nbr, __float_as_int(a0.w), 4 * ld * a1.nbr, __float_as_int(a1.w) | flag);
    rq[i] = make_int4(4 * ld * b0.nbr, __float_as_int(b0.w), 4 * ld * b1.nbr, __float_as_int(b1.w));
    rr[i] = make_int4(o0, o1, e_row + q0, e_row + q1);
  }
  for (int k = lt; kStaged && k < e_row; k += LG) {
    const CfAdj a = ldg_adj(g.r_oadj + eo0 + k), b = ldg_adj(g.r_iadj + ei0 + k);
    redge[k] = make_int2(4 * ld * a.nbr, __float_as_int(a.w));
    redge[e_row + k] = make_int2(4 * ld * b.nbr, __float_as_int(b.w));
  }
  for (int k = lt; kStaged && k < e_col; k += LG) {
    const CfAdj a = ldg_adj(g.c_oadj + co0 + k), b = ldg_adj(g.c_iadj + ci0 + k);
    cedge[k] = make_int2(4 * a.nbr, __float_as_int(a.w));
    cedge[e_col + k] = make_int2(4 * b.nbr, __float_as_int(b.w));
  }
  for (int k = lt; kStaged && k <= n_col; k += LG) {
    cptr[k] = __ldg(g.c_optr + k) - co0;
    cptr[n_col + 1 + k] = e_col + __ldg(g.c_iptr + k) - ci0;
  }
  // the columns with further neighbours, in index order (warp 0 of this CTA)
  int* nbcp = reinterpret_cast<int*>(align_up(reinterpret_cast<size_t>(cptr + 2 * (n_col + 1)), 16));
  int16_t* bcol = reinterpret_cast<int16_t*>(nbcp + 4);
  // and, for the busy-column sums, the sub-slot table (lane 0 of warp 0):
  // nbcp = {busy columns, sub-slots, slots, 0}; 0 sub-slots when the table
  // does not fit, and sweep_busy then takes those entries directly
  int2* bsub = reinterpret_cast<int2*>(align_up(reinterpret_cast<size_t>(bcol + n_col), 16));
  int* bslot = reinterpret_cast<int*>(bsub + kBusySubs);
  float* bpw = reinterpret_cast<float*>(bslot + kBusySlots) + loc.warp() * kBusySlots;
  if (kStaged && lt < 32) {
    int cnt = 0;
    for (int b = 0; b < n_col; b += 32) {
      const int j = b + lt;
      const bool x = j < n_col && (__ldg(g.c_optr + j + 1) - __ldg(g.c_optr + j) > 2 ||
                                   __ldg(g.c_iptr + j + 1) - __ldg(g.c_iptr + j) > 2);
      const unsigned msk = __ballot_sync(0xffffffffu, x);
      if (x) bcol[cnt + __popc(msk & ((1u << lt) - 1u))] = (int16_t)j;
      cnt += __popc(msk);
    }
    __syncwarp();
    if (lt == 0) {
      int ns = 0;
      bool fit = 2 * cnt <= kBusySlots;
      for (int b = 0; fit && b < cnt; ++b) {
        const int j = bcol[b];
        const int r0[2] = {__ldg(g.c_optr + j) - co0, e_col + __ldg(g.c_iptr + j) - ci0};
        const int r1[2] = {__ldg(g.c_optr + j + 1) - co0, e_col + __ldg(g.c_iptr + j + 1) - ci0};
        for (int d = 0; fit && d < 2; ++d) {
          const int first = ns;
          for (int e = r0[d]; e < r1[d]; e += 8) {
            if (ns == kBusySubs) {
              fit = false;
              break;
            }
            bsub[ns++] = make_int2(e, min(8, r1[d] - e) | ((2 * b + d) << 8));
          }
          bslot[2 * b + d] = first | ((ns - first) << 16);
        }
      }
      nbcp[0] = cnt;
      nbcp[1] = fit ? ns : 0;
      nbcp[2] = 2 * cnt;
    }
  }
  grp.sync();  // staged lists (this CTA) and row norms (the team) visible
  const int nbc = kStaged ? nbcp[0] : 0;
  const int nsub = kStaged ? nbcp[1] : 0;
  float* T = reinterpret_cast<float*>(ms + n_row + 2 * n_col);

  // The prologue visits entries in row-major order, team thread t taking t,
  // t + G, ...: the team sweeps a narrow band of rows at a time.  (i, j) of
  // the next entry follow without a division.  The iterations run by strips
  // (sweep_strips, sweep_busy).

  // a3: E, |E|, Ehat = X_0
  float ss = 0.f;
  for_entries(n_row, n_col, ld, t, G, [&](int i, int j, size_t off) {
    const float* bcol = g.c_attr + (size_t)j * cx.Fp;
    const float den = rn[i] * rn[n_row + j];
    const float e = den > 0.f ? attr_dot(g.r_attr + (size_t)i * cx.Fp, bcol, cx.om, cx.Fp) / den : 0.f;
    ehb[off] = e;
    ss = fmaf(e, e, ss);
  });
  const float tot = grp.sum(ss, 0);
  const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  const float uni = 1.0f / sqrtf((float)n_row * (float)n_col);
  const float cb = 1.f - cx.alpha;
  for_entries(n_row, n_col, ld, t, G, [&](int, int, size_t off) {
    const float eh = tot > 0.f ? ehb[off] * inv : uni;
    buf0[off] = eh;
    ehb[off] = cb * eh;
  });
  grp.sync();

  // a4: K renormalised iterations, one barrier each
  const StripPlan sp = strip_plan(n_row, n_col, G);
  float sk = 1.f;
  for (int k = 0; k < cx.K; ++k) {
    const char* cur = reinterpret_cast<const char*>((k & 1) ? buf1 : buf0);
    float* nxt = (k & 1) ? buf0 : buf1;
    const float ca = 0.5f * cx.alpha * sk;
    if (kStaged) {
      ss = sweep_strips<U>(sp, t, G, n_row, n_col, ld, cur, nxt, ehb, ca, ra, rq, rr, redge, cedge, cptr);
      if (nsub > 0) {
        bsum_rows(grp.warp(), grp.nwarps(), t & 31, n_row, ld, cur, nsub, bsub, nbcp[2], bslot, cedge, bpw, T);
        grp.sync();  // T complete
        ss += bsum_entries(nbc, bcol, t, G, n_row, ld, nxt, ehb, ca, ra, rq, rr, redge, T);
      } else {
        ss += sweep_busy(nbc, bcol, t, G, n_row, n_col, ld, cur, nxt, ehb, ca, ra, rq, rr, redge, cedge, cptr);
      }
    } else {
      ss = 0.f;
      for_entries(n_row, n_col, ld, t, G, [&](int i, int j, size_t off) {
        const float z = gather_g(reinterpret_cast<const float*>(cur), ld, g, i, j);
        const float y = fmaf(ca, z, ehb[off]);
        nxt[off] = y;
        ss = fmaf(y, y, ss);
      });
    }
    const float yy = grp.sum(ss, (k + 1) & 1);
    sk = cx.norm_mode == 0 ? 1.0f / sqrtf(yy) : 1.f;
  }
  float* Xs = (cx.K & 1) ? buf1 : buf0;
  if (sk != 1.f) for_entries(n_row, n_col, ld, t, G, [&](int, int, size_t off) { Xs[off] *= sk; });
  grp.sync();
  if (cx.X) store_x(grp, cx, g, Xs, n_col);
  if (cx.scores || cx.match) {
    int32_t* mo = cx.match ? cx.match + cx.m_off[g.p] : nullptr;
    float sc;
    if constexpr (kStaged && std::is_same<Grp, Group>::value)  // one CTA: the state in its shared memory
      sc = greedy_g(grp, Xs, n_row, n_col, ehb, region, mo, cx.hdr, g.p);
    else
      sc = greedy<int32_t>(grp, Xs, n_col, n_row, n_col, 0, ms, ms + n_row, ms + n_row + n_col, mo, cx.hdr, g.p);
    if (cx.scores && t == 0) cx.scores[g.p] = sc;
  }
  grp.sync();
}

// Rows per batch of the global tier's sweep: as many loads in flight as the
// thread count's register budget holds (128, 80 and 64 registers).
constexpr int strip_u(int NT) { return NT <= 512 ? 8 : (NT <= 768 ? 4 : 2); }

// Whether a global-class pair's graphs can be staged in the CTA's shared memory.
__device__ __forceinline__ bool staged_fits(const Geo& g, int region) {
  const int e_row = __ldg(g.r_optr + g.na) - __ldg(g.r_optr);
  const int e_col = __ldg(g.c_optr + g.nb) - __ldg(g.c_optr);
  return 48 * (size_t)g.na + 16 * (size_t)(e_row + e_col) + 8 * (size_t)(g.nb + 2) + 32 + 2 * (size_t)g.nb + 16 +
             8 * kBusySubs + 4 * kBusySlots + 32 * 4 * kBusySlots <=
         (size_t)region;
}

// Per-CTA setup, done by thread 0 into shared memory (so the pack views do
// not occupy registers in the hot loop): pack views, workspace pointers,
// omega (validated).  Returns false on every thread if the call is invalid.
__device__ __forceinline__ bool make_ctx(const CallArgs& a, float* s_om, Ctx& cx, int* s_ok) {
  if (threadIdx.x == 0) {
    cx.A = load_pack(a.pack_a);
    cx.B = load_pack(a.pack_b);
    const WsLayout L = ws_layout(a.P);
    cx.hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
    cx.queue = reinterpret_cast<const uint32_t*>(a.ws + L.queue);
    cx.x_off = reinterpret_cast<const int64_t*>(a.ws + L.x_off);
    cx.m_off = reinterpret_cast<const int64_t*>(a.ws + L.m_off);
    cx.scratch = a.ws + L.scratch;
    cx.scratch_bytes = a.ws_bytes > L.scratch ? a.ws_bytes - L.scratch : 0;
    cx.def_rk = nullptr;
    cx.def_rkey = nullptr;
    cx.def_list = nullptr;
    if (cx.hdr->defer) {  // the scratch slots end where the deferred-steps area starts
      const uint64_t off = cx.hdr->defer_off;
      const int64_t xt = cx.hdr->x_total;
      cx.scratch_bytes = off > L.scratch ? off - L.scratch : 0;
      cx.def_rk = reinterpret_cast<int16_t*>(a.ws + off);
      cx.def_rkey = reinterpret_cast<uint32_t*>(a.ws + off + align_up(2 * (size_t)xt, kAlign));
      cx.def_list = reinterpret_cast<uint32_t*>(a.ws + off + align_up(2 * (size_t)xt, kAlign) +
                                                align_up(4 * (size_t)xt, kAlign));
    }
    cx.pairs = a.pairs;
    cx.alpha = a.alpha;
    cx.K = a.K;
    cx.norm_mode = a.norm_mode;
    cx.X = a.X;
    cx.scores = a.scores;
    cx.match = a.match;
    cx.F = cx.A.F;
    cx.Fp = cx.A.F_pad;
    cx.ranked = a.ranked;
    cx.om = s_om;
    cx.sqom = s_om + kMaxF;
    *s_ok = (cx.A.F == cx.B.F && cx.A.F_pad == cx.B.F_pad) ? 1 : 0;
    if (!*s_ok && blockIdx.x == 0) set_status(cx.hdr, 1 /* CF_ERR_INVALID_ARG */, -1);
  }
  __syncthreads();
  if (!*s_ok) return false;
  if (threadIdx.x < kMaxF) {
    const float v = threadIdx.x < cx.F ? a.omega[threadIdx.x] : 0.f;
    s_om[threadIdx.x] = v;
    s_om[kMaxF + threadIdx.x] = sqrtf(v);
    if (!(v >= 0.f && v <= 3.0e38f) && blockIdx.x == 0) set_status(cx.hdr, 6 /* CF_ERR_NUMERIC */, threadIdx.x);
  }
  __syncthreads();
  return true;
}

// The persistent kernel's shapes: NT threads, one CTA per SM, 220 KB of
// dynamic shared memory split 1 / 2 / 4 / 8 / (NT/32) ways for the five group
// levels.
constexpr size_t kFwdSmem = 225280;
template <int NT>
__host__ __device__ constexpr ClassCfg fwd_cfg(int min_cls = kClassWarp, int ranked = 0, int cluster = 0) {
  return ClassCfg{NT,
                  (int)kFwdSmem,
                  (int)kFwdSmem / 2,
                  (int)kFwdSmem / 4,
                  (int)kFwdSmem / 8,
                  ((int)kFwdSmem / (NT / 32)) & ~15,
                  min_cls,
                  ranked,
                  cluster};
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) fwd_batched_kernel(CallArgs a, int per_pair, int pp_slot) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) float s_om[2 * kMaxF];  // omega, then sqrt(omega)
  __shared__ Ctx s_cx;
  __shared__ int s_ok;
  __shared__ uint32_t s_p[1 + 2 + 4 + 8 + NT / 32];  // queue positions: CTA, half, quarter, eighth groups, warps
  // per-warp partials, two parities, of the CTA group, then the half,
  // quarter and eighth groups: 2 * NT / 32 entries per level
  __shared__ float s_redf[4][2 * NT / 32];
  __shared__ int s_redi[4][2 * NT / 32];
  if (!make_ctx(a, s_om, s_cx, &s_ok)) return;
  const Ctx& cx = s_cx;
  const bool single = per_pair >= 0;  // the plain form: one launch runs exactly one pair on the whole CTA
  // the per-pair form keeps every pair on the whole CTA
  const ClassCfg cc = fwd_cfg<NT>(single ? (int)kClassCta : a.min_cls, a.ranked);
  const int t = threadIdx.x;
  const Group cta{t, NT, 0, s_redf[0], s_redi[0]};

  uint32_t n[kNumClasses];
  for (int c = 0; c < kNumClasses; ++c) n[c] = single ? 0u : cx.hdr->n_class[c];
  // global class: whole CTA, one scratch slot per CTA (with the cluster tier
  // on, the cluster kernel has run these pairs)
  if (n[kClassGlobal] > 0 && a.cluster < 2) {
    const uint64_t need = cx.hdr->slot_need;
    const uint64_t nslots = need ? cx.scratch_bytes / need : 0;
    if (nslots == 0) {
      if (blockIdx.x == 0 && t == 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    } else if (blockIdx.x < nslots &&
               bounds_ok(cx.hdr, ((size_t)blockIdx.x + 1) * need <= cx.scratch_bytes, kSiteFwdSlot)) {
      float* slot = reinterpret_cast<float*>(cx.scratch + (size_t)blockIdx.x * need);
      for (;;) {
        if (t == 0) s_p[0] = atomicAdd(&cx.hdr->q_next[kClassGlobal], 1u);
        __syncthreads();
        const uint32_t q = s_p[0];
        __syncthreads();
        if (q >= n[kClassGlobal]) break;
        {
          const Geo g = make_geo(cx, (int)cx.queue[q], cc);
          if (staged_fits(g, cc.z_cta))
            run_pair_g<true, strip_u(NT)>(cx, g, cta, cta, slot, smem);
          else
            run_pair_g<false, 1>(cx, g, cta, cta, slot, smem);
        }
      }
    }
  }
  // shared-memory classes, one level after the other: the whole CTA, then
  // two half groups (named barriers 5..6), four quarter groups (named
  // barriers 1..4), eight eighth groups (named barriers 7..14), then single
  // warps.  Each level is a sub-partition of the
  // previous one's region, and every group ends a pair with its own barrier,
  // so no CTA-wide barrier sits between levels.
  uint32_t qbase = n[kClassGlobal];
  for (int level = kClassCta; level <= cc.min_cls; ++level) {
    Group grp = cta;
    unsigned char* region = smem;
    int slot = 0;
    if (level == kClassHalf) {
      const int hg = t / (NT / 2);
      grp = Group{t % (NT / 2), NT / 2, 5 + hg, s_redf[1] + hg * (NT / 32), s_redi[1] + hg * (NT / 32)};
      region = smem + (size_t)hg * cc.z_half;
      slot = 1 + hg;
    } else if (level == kClassQuarter) {
      const int qg = t / (NT / 4);
      grp = Group{t % (NT / 4), NT / 4, 1 + qg, s_redf[2] + qg * (NT / 64), s_redi[2] + qg * (NT / 64)};
      region = smem + (size_t)qg * cc.z_qtr;
      slot = 3 + qg;
    } else if (level == kClassEighth) {
      const int eg = t / (NT / 8);
      grp = Group{t % (NT / 8), NT / 8, 7 + eg, s_redf[3] + eg * (NT / 128), s_redi[3] + eg * (NT / 128)};
      region = smem + (size_t)eg * cc.z_8th;
      slot = 7 + eg;
    } else if (level == kClassWarp) {
      grp = Group{t & 31, 32, -1, nullptr, nullptr};
      region = smem + (size_t)(t >> 5) * cc.z_wrp;
      slot = 15 + (t >> 5);
    }
    const uint32_t count = single ? 1u : n[level];
    for (;;) {
      if (grp.rank == 0) s_p[slot] = single ? 0u : atomicAdd(&cx.hdr->q_next[level], 1u);
      grp.sync();
      const uint32_t q = s_p[slot];
      grp.sync();
      if (q >= count) break;
      if (single && grp.rank == 0) s_p[slot] = 1u;  // the next pull ends the loop
      const Geo g = make_geo(cx, single ? per_pair : (int)cx.queue[qbase + q], cc);
      if (g.s.cls == kClassGlobal) {  // only in the plain form: the scratch slot of its stream
        const size_t need = pp_slot > 0 ? (size_t)cx.hdr->slot_need : 0;
        float* pslot = reinterpret_cast<float*>(cx.scratch + (size_t)pp_slot * need);
        if (global_slot_bytes(g.na, g.nb) + (size_t)pp_slot * need > cx.scratch_bytes) {
          if (t == 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, per_pair);
        } else {
          if (staged_fits(g, cc.z_cta))
            run_pair_g<true, strip_u(NT)>(cx, g, cta, cta, pslot, smem);
          else
            run_pair_g<false, 1>(cx, g, cta, cta, pslot, smem);
        }
        break;
      }
      run_pair_s(cx, g, grp, region, group_region(level, cc));
      if (single) break;
    }
    qbase += single ? 0u : n[level];
  }
}

// ---------------------------------------------------------------------------
// The cluster tier: a pair too large for one CTA's shared memory is split by
// rows over the C CTAs of a thread-block cluster.  CTA r holds rows
// [r S, r S + S) (S = ceil(n_row / C)) of (1 - alpha) Ehat and of both
// iterates, the first-two / further neighbour lists of its rows, and the
// whole column graph.  The row lists name each neighbour row u by the 32-bit
// shared::cluster address of row u in its owner's buffer 0, so a gather
// reads the owner's shared memory directly (ld.shared::cluster): one code
// path for local and remote rows.  One cluster barrier per iteration (inside
// the cluster-wide norm reduction) separates the reads of Y_k from the
// writes of Y_{k+2} into the same buffer.  X_K is then written to the
// cluster's scratch slot and CTA 0 runs the greedy matching on it.

__device__ __noinline__ void run_pair_c(const Ctx& cx, const Geo& g, const Group& grp, int C, int rank, float* slot,
                                        unsigned char* region, ClState& st) {
  const Shape& s = g.s;
  const int t = grp.rank, G = grp.size;
  const int ld = s.ld;
  const int slab = ceil_div(s.n_row, C);
  const int i0 = rank * slab;
  const int rows = max(0, min(s.n_row, i0 + slab) - i0);
  const int nn = slab * ld;
  float* ehb = reinterpret_cast<float*>(region);
  float* buf0 = ehb + nn;
  float* buf1 = buf0 + nn;
  int4* ra = reinterpret_cast<int4*>(region + align_up(12 * (size_t)nn, 16));
  int4* rq = ra + slab;
  int4* rr = rq + slab;
  int2* redge = reinterpret_cast<int2*>(rr + slab);
  // Row u (of the whole row graph) as the gathers address it: for a row whose
  // neighbours all lie in this CTA's slab, the byte offset of u in this CTA's
  // buffer (plain shared loads); otherwise the cluster address of u in its
  // owner's buffer 0 (ld.shared::cluster), and A.y of the row is flagged.
  auto raddr = [&](int u, bool remote) -> int {
    if (!remote) return (u - i0) * ld * 4;
    const int o = u / slab;
    return (int)(st.rbase[o] + 4u * (uint32_t)nn + 4u * (uint32_t)((u - o * slab) * ld));
  };

  const int eo0 = __ldg(g.r_optr), ei0 = __ldg(g.r_iptr);
  const int so0 = __ldg(g.r_optr + i0) - eo0, so1 = __ldg(g.r_optr + i0 + rows) - eo0;
  const int si0 = __ldg(g.r_iptr + i0) - ei0, si1 = __ldg(g.r_iptr + i0 + rows) - ei0;
  const int n_so = so1 - so0, n_si = si1 - si0;
  const int co0 = __ldg(g.c_optr), ci0 = __ldg(g.c_iptr);
  const int e_col = __ldg(g.c_optr + s.n_col) - co0;
  int2* cedge = redge + (n_so + n_si);
  int* cptr = reinterpret_cast<int*>(cedge + 2 * e_col);
  for (int k = t; k < e_col; k += G) {
    const CfAdj a = ldg_adj(g.c_oadj + co0 + k), b = ldg_adj(g.c_iadj + ci0 + k);
    cedge[k] = make_int2(4 * a.nbr, __float_as_int(a.w));
    cedge[e_col + k] = make_int2(4 * b.nbr, __float_as_int(b.w));
  }
  for (int k = t; k <= s.n_col; k += G) {
    cptr[k] = __ldg(g.c_optr + k) - co0;
    cptr[s.n_col + 1 + k] = e_col + __ldg(g.c_iptr + k) - ci0;
  }
  for (int lr = t; lr < rows; lr += G) {
    const int i = i0 + lr;
    const int o0 = __ldg(g.r_optr + i) - eo0, o1 = __ldg(g.r_optr + i + 1) - eo0;
    const int q0 = __ldg(g.r_iptr + i) - ei0, q1 = __ldg(g.r_iptr + i + 1) - ei0;
    bool remote = false;
    for (int e = o0; e < o1; ++e) {
      const int u = __ldg(&g.r_oadj[eo0 + e].nbr);
      remote |= u < i0 || u >= i0 + slab;
    }
    for (int e = q0; e < q1; ++e) {
      const int u = __ldg(&g.r_iadj[ei0 + e].nbr);
      remote |= u < i0 || u >= i0 + slab;
    }
    const CfAdj z{i0, 0.f};  // padding: a valid row of this CTA's slab, weight 0
    const CfAdj a0 = o1 > o0 ? ldg_adj(g.r_oadj + eo0 + o0) : z, a1 = o1 > o0 + 1 ? ldg_adj(g.r_oadj + eo0 + o0 + 1) : z;
    const CfAdj b0 = q1 > q0 ? ldg_adj(g.r_iadj + ei0 + q0) : z, b1 = q1 > q0 + 1 ? ldg_adj(g.r_iadj + ei0 + q0 + 1) : z;
    const int flag = (o1 - o0 > 2 || q1 - q0 > 2) ? (int)0x80000000 : 0;
    const int rflag = remote ? (int)0x80000000 : 0;
    ra[lr] = make_int4(raddr(a0.nbr, remote), __float_as_int(a0.w) | rflag, raddr(a1.nbr, remote),
                       __float_as_int(a1.w) | flag);
    rq[lr] = make_int4(raddr(b0.nbr, remote), __float_as_int(b0.w), raddr(b1.nbr, remote), __float_as_int(b1.w));
    rr[lr] = make_int4(o0 - so0, o1 - so0, n_so + q0 - si0, n_so + q1 - si0);
    // this row's full lists, addressed the same way
    for (int e = o0; e < o1; ++e) {
      const CfAdj a = ldg_adj(g.r_oadj + eo0 + e);
      redge[e - so0] = make_int2(raddr(a.nbr, remote), __float_as_int(a.w));
    }
    for (int e = q0; e < q1; ++e) {
      const CfAdj b = ldg_adj(g.r_iadj + ei0 + e);
      redge[n_so + e - si0] = make_int2(raddr(b.nbr, remote), __float_as_int(b.w));
    }
  }
  for (int lr = t; lr < rows; lr += G) buf1[lr] = attr_norm(g.r_attr + (size_t)(i0 + lr) * cx.Fp, cx.om, cx.Fp);
  const bool act = t < s.R * s.n_col;
  const int j = act ? t % s.n_col : 0;
  const int r0 = act ? t / s.n_col : 0;
  const int Mt = (act && rows > r0) ? ceil_div(rows - r0, s.R) : 0;
  const int step = s.R * ld;
  const int off0 = r0 * ld + j;
  const float* bcol = g.c_attr + (size_t)j * cx.Fp;
  const float cj = attr_norm(bcol, cx.om, cx.Fp);
  __syncthreads();

  // a3: E over the slab, |E|_F over the cluster, Ehat = X_0
  float ss = 0.f;
  for (int m = 0, lr = r0, off = off0; m < Mt; ++m, lr += s.R, off += step) {
    const float dot = attr_dot(g.r_attr + (size_t)(i0 + lr) * cx.Fp, bcol, cx.om, cx.Fp);
    const float den = buf1[lr] * cj;
    const float e = den > 0.f ? dot / den : 0.f;
    ehb[off] = e;
    ss = fmaf(e, e, ss);
  }
  const float tot = cl_sum(ss, 0, st, C);
  const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  const float uni = 1.0f / sqrtf((float)s.n_row * (float)s.n_col);
  const float cb = 1.f - cx.alpha;
  for (int m = 0, off = off0; m < Mt; ++m, off += step) {
    const float eh = tot > 0.f ? ehb[off] * inv : uni;
    buf0[off] = eh;
    ehb[off] = cb * eh;
  }
  cl_sync();  // every slab of Y_0 (and the staged lists) visible
  const ColPad cl = load_col(cptr, cedge, s.n_col, j);

  // a4: K renormalised iterations, one cluster barrier each
  float sk = 1.f;
  for (int k = 0; k < cx.K; ++k) {
    const ClusterY cur{(k & 1) ? 4u * (uint32_t)nn : 0u};
    const char* lcur = reinterpret_cast<const char*>((k & 1) ? buf1 : buf0);
    float* nxt = (k & 1) ? buf0 : buf1;
    const float ca = 0.5f * cx.alpha * sk;
    ss = 0.f;
    for (int m = 0, lr = r0, off = off0; m < Mt; ++m, lr += s.R, off += step) {
      const int4 A = ra[lr], Q = rq[lr];
      float z;
      if (A.y >= 0) {  // every neighbour row in this CTA: plain shared loads
        z = gather_fast(lcur, A, Q, cl);
        if (A.w < 0 || cl.flag) {
          const int4 R4 = rr[lr];
          if (A.w < 0) z += row_extra(lcur, R4, redge, cl);
          if (cl.flag) z += col_extra(lcur, A, Q, R4, redge, cedge, cptr, s.n_col, j);
        }
      } else {
        z = gather_fast(cur, A, Q, cl);
        if (A.w < 0 || cl.flag) {
          const int4 R4 = rr[lr];
          if (A.w < 0) z += row_extra(cur, R4, redge, cl);
          if (cl.flag) z += col_extra(cur, A, Q, R4, redge, cedge, cptr, s.n_col, j);
        }
      }
      const float y = fmaf(ca, z, ehb[off]);
      nxt[off] = y;
      ss = fmaf(y, y, ss);
    }
    const float yy = cl_sum(ss, (k + 1) & 1, st, C);
    sk = cx.norm_mode == 0 ? 1.0f / sqrtf(yy) : 1.f;
  }
  const float* Xs = (cx.K & 1) ? buf1 : buf0;

  // X_K to the scratch slot (row-graph orientation, stride n_col) and, if
  // asked, to the caller's n_a x n_b output
  float* xo = cx.X ? cx.X + cx.x_off[g.p] : nullptr;
  for (int m = 0, lr = r0, off = off0; m < Mt; ++m, lr += s.R, off += step) {
    const float x = Xs[off] * sk;
    const int i = i0 + lr;
    slot[(size_t)i * s.n_col + j] = x;
    if (xo) xo[s.tr ? (size_t)j * s.n_row + i : (size_t)i * s.n_col + j] = x;
  }
  cl_sync();  // the whole X_K is in the slot
  if (cx.scores || cx.match) {
    // the greedy rounds on the whole cluster: rows and columns spread over
    // every warp of every CTA, the matching state in the slot
    const ClGroup cg{rank * G + t, C * G, C, &st};
    int32_t* ms = reinterpret_cast<int32_t*>(slot + (size_t)s.n_row * s.n_col);
    int32_t* mo = cx.match ? cx.match + cx.m_off[g.p] : nullptr;
    const float sc = greedy<int32_t>(cg, slot, s.n_col, s.n_row, s.n_col, s.tr, ms, ms + s.n_row,
                                     ms + s.n_row + s.n_col, mo, cx.hdr, g.p);
    if (cx.scores && cg.rank == 0) cx.scores[g.p] = sc;
  }
}

// Persistent clusters drain the cluster-class queue (after the global and
// shared-memory classes in the plan's queue): CTA 0 of a cluster pulls a
// pair and every CTA reads the index from its shared memory.  Each cluster
// uses the scratch slot of its index.
template <int NT>
__global__ void __launch_bounds__(NT, 1) fwd_cluster_kernel(CallArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) float s_om[2 * kMaxF];  // omega, then sqrt(omega)
  __shared__ Ctx s_cx;
  __shared__ int s_ok;
  __shared__ ClState st;
  __shared__ float s_redf[64];
  __shared__ int s_redi[64];
  if (!make_ctx(a, s_om, s_cx, &s_ok)) return;  // same outcome on every CTA (depends on the packs only)
  const Ctx& cx = s_cx;
  const int t = threadIdx.x;
  const int C = (int)cl_size(), rank = (int)cl_rank();
  const uint32_t cid = cl_index();
  const uint32_t n_cl = cx.hdr->n_class[kClassCluster], n_gl = cx.hdr->n_class[kClassGlobal];
  if (n_cl == 0 && n_gl == 0) return;
  const uint64_t need = cx.hdr->slot_need;
  const uint64_t nslots = need ? cx.scratch_bytes / need : 0;
  if (nslots == 0) {
    if (cid == 0 && rank == 0 && t == 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    return;
  }
  if (cid >= nslots) return;  // the whole cluster
  const ClassCfg cc = fwd_cfg<NT>(a.min_cls, a.ranked, C);
  uint32_t qbase = 0;
  for (int c = 0; c < kClassCluster; ++c) qbase += cx.hdr->n_class[c];
  if (t < C) {
    st.rbase[t] = cl_map(smem, t);
    st.paddr[t] = cl_map(st.part, t);
    st.piaddr[t] = cl_map(st.parti, t);
  }
  if (t == 0) st.qaddr = cl_map(&st.q, 0);
  __syncthreads();
  float* slot = reinterpret_cast<float*>(cx.scratch + (size_t)cid * need);
  const Group cta{t, NT, 0, s_redf, s_redi};
  // the global class (too large for the cluster's shared memory): the whole
  // cluster sweeps the pair's L2-resident slot
  const ClGroup team{rank * NT + t, C * NT, C, &st};
  for (;;) {
    if (rank == 0 && t == 0) st.q = atomicAdd(&cx.hdr->q_next[kClassGlobal], 1u);
    cl_sync();
    const uint32_t q = cl_ld_u32(st.qaddr);
    cl_sync();  // CTA 0 overwrites q only after every CTA has read it
    if (q >= n_gl) break;
    const Geo g = make_geo(cx, (int)cx.queue[q], cc);
    if (staged_fits(g, cc.z_cta))
      run_pair_g<true, strip_u(NT)>(cx, g, cta, team, slot, smem);
    else
      run_pair_g<false, 1>(cx, g, cta, team, slot, smem);
  }
  for (;;) {
    if (rank == 0 && t == 0) st.q = atomicAdd(&cx.hdr->q_next[kClassCluster], 1u);
    cl_sync();
    const uint32_t q = cl_ld_u32(st.qaddr);
    cl_sync();  // CTA 0 overwrites q only after every CTA has read it
    if (q >= n_cl) break;
    const Geo g = make_geo(cx, (int)cx.queue[qbase + q], cc);
    run_pair_c(cx, g, cta, C, rank, slot, smem, st);
  }
}

// The deferred sequential steps of the greedy matching (matching policy 3).
// The forward ranked each resident pair's lists in its group and left them
// in the workspace (pair p's at x_off[p]), initialised its matching to -1 and
// listed the pair (index | orientation << 31); here every warp takes listed
// pairs one after another and runs the steps of greedy_seq on them, so that
// a group of the forward is not held by one warp's chain of steps.  The dead
// flags live in the warp's shared memory.
constexpr int kDefNT = 256;

__global__ void __launch_bounds__(kDefNT) match_deferred_kernel(CallArgs a) {
  __shared__ unsigned char s_dead[kDefNT / 32][kSeqMaxLists];
  __shared__ PackView sA, sB;
  const WsLayout L = ws_layout(a.P);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
  if (!hdr->defer) return;  // the forward matched every pair itself
  if (threadIdx.x == 0) {
    sA = load_pack(a.pack_a);
    sB = load_pack(a.pack_b);
  }
  __syncthreads();
  const uint64_t off = hdr->defer_off;
  const int64_t xt = hdr->x_total;
  const int16_t* def_rk = reinterpret_cast<const int16_t*>(a.ws + off);
  const uint32_t* def_rkey = reinterpret_cast<const uint32_t*>(a.ws + off + align_up(2 * (size_t)xt, kAlign));
  const uint32_t* def_list = reinterpret_cast<const uint32_t*>(a.ws + off + align_up(2 * (size_t)xt, kAlign) +
                                                               align_up(4 * (size_t)xt, kAlign));
  const int64_t* x_off = reinterpret_cast<const int64_t*>(a.ws + L.x_off);
  const int64_t* m_off = reinterpret_cast<const int64_t*>(a.ws + L.m_off);
  const uint32_t n = hdr->n_def;
  const int lane = threadIdx.x & 31;
  unsigned char* dead = s_dead[threadIdx.x >> 5];
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(&hdr->q_def, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= n) break;
    const uint32_t ent = def_list[q];
    const int p = (int)(ent & 0x7fffffffu), tr = (int)(ent >> 31);
    const int pa = __ldg(a.pairs + 2 * p), pb = __ldg(a.pairs + 2 * p + 1);
    const int na = __ldg(sA.node_off + pa + 1) - __ldg(sA.node_off + pa);
    const int nb = __ldg(sB.node_off + pb + 1) - __ldg(sB.node_off + pb);
    const int n_row = tr ? nb : na, n_col = tr ? na : nb;
    const bool rows = n_col <= n_row;
    const int nl = rows ? n_row : n_col, len = rows ? n_col : n_row;
    const bool swap = rows == (tr != 0);
    for (int e = lane; e < len; e += 32) dead[e] = 0;
    __syncwarp();
    const int16_t* rk = def_rk + x_off[p];
    const uint32_t* rkey = def_rkey + x_off[p];
    int32_t* mo = a.match ? a.match + m_off[p] : nullptr;
    const int Rn = (nl + 31) >> 5;
    float sc;
    if (Rn <= 1)
      sc = greedy_seq_steps<1>(lane, swap, nl, len, rk, rkey, dead, mo, hdr, p);
    else if (Rn <= 2)
      sc = greedy_seq_steps<2>(lane, swap, nl, len, rk, rkey, dead, mo, hdr, p);
    else if (Rn <= 4)
      sc = greedy_seq_steps<4>(lane, swap, nl, len, rk, rkey, dead, mo, hdr, p);
    else
      sc = greedy_seq_steps<8>(lane, swap, nl, len, rk, rkey, dead, mo, hdr, p);
    if (a.scores && lane == 0) a.scores[p] = sc;
    __syncwarp();
  }
}

// cf_match on caller-given matrices: one CTA per pair, matching state in
// shared memory (int16, up to kMaxBlocks rows and columns).
constexpr int kMatchNT = 512;

__global__ void __launch_bounds__(kMatchNT) match_only_kernel(CallArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float redf[64];
  __shared__ int redi[64];
  const PackView A = load_pack(a.pack_a), B = load_pack(a.pack_b);
  const WsLayout L = ws_layout(a.P);
  const int64_t* x_off = reinterpret_cast<const int64_t*>(a.ws + L.x_off);
  const int64_t* m_off = reinterpret_cast<const int64_t*>(a.ws + L.m_off);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
  int16_t* ms = reinterpret_cast<int16_t*>(smem);
  const Group grp{(int)threadIdx.x, kMatchNT, 0, redf, redi};
  for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
    const int pa = a.pairs[2 * p], pb = a.pairs[2 * p + 1];
    if (pa < 0 || pa >= A.n_cfgs || pb < 0 || pb >= B.n_cfgs) continue;  // recorded by the plan
    const int na = A.node_off[pa + 1] - A.node_off[pa];
    const int nb = B.node_off[pb + 1] - B.node_off[pb];
    const float* X = a.X_in + x_off[p];
    int32_t* mo = a.match ? a.match + m_off[p] : nullptr;
    const float sc = greedy<int16_t>(grp, X, nb, na, nb, 0, ms, ms + na, ms + na + nb, mo, hdr, p);
    if (a.scores && threadIdx.x == 0) a.scores[p] = sc;
    __syncthreads();
  }
}

// Per device: the side streams and events of the plain form spread over
// streams (CF_FLAG_PER_PAIR_STREAMS), created on first use.
struct PerPairStreams {
  cudaStream_t side[kPerPairStreams] = {};
  cudaEvent_t fork = nullptr, join[kPerPairStreams] = {};
  std::mutex mu;  // one fork / join sequence at a time (the events are shared)
};

cudaError_t per_pair_streams(PerPairStreams** out) {
  static DeviceOnce once;
  static PerPairStreams devs[kMaxDevices];
  int dev = 0;
  const cudaError_t e = once.run(
      [](int d) {
        PerPairStreams& ps = devs[d];
        cudaError_t r = cudaEventCreateWithFlags(&ps.fork, cudaEventDisableTiming);
        for (int k = 0; k < kPerPairStreams && r == cudaSuccess; ++k) {
          r = cudaStreamCreateWithFlags(&ps.side[k], cudaStreamNonBlocking);
          if (r == cudaSuccess) r = cudaEventCreateWithFlags(&ps.join[k], cudaEventDisableTiming);
        }
        return r;
      },
      &dev);
  *out = e == cudaSuccess ? &devs[dev] : nullptr;
  return e;
}

// Per device: the kernel's shared-memory limit and the SM count (the grid).
template <int NT>
cudaError_t fwd_init(int* n_sm) {
  static DeviceOnce once;
  static int sms[kMaxDevices];
  int dev = 0;
  const cudaError_t e = once.run(
      [](int d) {
        const cudaError_t r =
            cudaFuncSetAttribute(fwd_batched_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        sms[d] = sm_count_of(d);
        return r != cudaSuccess ? r : (sms[d] > 0 ? cudaSuccess : cudaErrorInvalidDevice);
      },
      &dev);
  *n_sm = e == cudaSuccess ? sms[dev] : 0;
  return e;
}

template <int NT>
cudaError_t launch_fwd(const CallArgs& a, bool per_pair, cudaStream_t s) {
  int n_sm = 0;
  cudaError_t e = fwd_init<NT>(&n_sm);
  if (e != cudaSuccess) return e;
  if (per_pair && a.pp_streams > 1) {
    // the plain form spread over side streams forked from s and joined back:
    // pair p on stream p mod S, with that stream's scratch slot
    PerPairStreams* ps = nullptr;
    e = per_pair_streams(&ps);
    if (e != cudaSuccess) return e;
    const int S = a.pp_streams < kPerPairStreams ? a.pp_streams : kPerPairStreams;
    std::lock_guard<std::mutex> lk(ps->mu);
    e = cudaEventRecord(ps->fork, s);
    for (int k = 0; k < S && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ps->side[k], ps->fork, 0);
    for (int p = 0; p < a.P && e == cudaSuccess; ++p)
      fwd_batched_kernel<NT><<<1, NT, kFwdSmem, ps->side[p % S]>>>(a, p, p % S);
    for (int k = 0; k < S && e == cudaSuccess; ++k) {
      e = cudaEventRecord(ps->join[k], ps->side[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ps->join[k], 0);
    }
    if (e != cudaSuccess) return e;
  } else if (per_pair) {
    for (int p = 0; p < a.P; ++p) fwd_batched_kernel<NT><<<1, NT, kFwdSmem, s>>>(a, p, 0);
  } else {
    fwd_batched_kernel<NT><<<n_sm, NT, kFwdSmem, s>>>(a, -1, 0);
  }
  return cudaGetLastError();
}

// Resident clusters of C CTAs of fwd_cluster_kernel<NT>, per device and C
// (queried once each; 0 if none fit).
template <int NT>
int resident_clusters(int C) {
  static std::mutex mu;
  static int known[kMaxDevices][kMaxCluster + 1];  // 0 unknown, else 1 + the count
  if (C < 2 || C > kMaxCluster) return 0;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (known[dev][C] > 0) return known[dev][C] - 1;
  int n = 0;
  if (cudaFuncSetAttribute(fwd_cluster_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) ==
          cudaSuccess &&
      cudaFuncSetAttribute(fwd_cluster_kernel<NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = kFwdSmem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, fwd_cluster_kernel<NT>, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  known[dev][C] = 1 + n;
  return n;
}

template <int NT>
cudaError_t launch_cluster(const CallArgs& a, cudaStream_t s) {
  const int C = a.cluster;
  const int n = resident_clusters<NT>(C);
  if (n <= 0) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(n * C, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = kFwdSmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fwd_cluster_kernel<NT>, a);
}

}  // namespace

int cluster_supported(int v, int C) {
  const int n = v == 1   ? resident_clusters<512>(C)
                : v == 2 ? resident_clusters<768>(C)
                         : resident_clusters<1024>(C);
  return n > 0 ? C : 0;
}

// Variants of the persistent forward kernel: 0 = 1024 threads (64 registers,
// 32 warps per SM), 1 = 512 threads (128 registers, 16 warps per SM), 2 = 768
// threads (80 registers, 24 warps per SM).
int num_fwd_variants() { return 3; }

ClassCfg fwd_class_cfg(int v, int min_cls, int ranked, int cluster) {
  return v == 1   ? fwd_cfg<512>(min_cls, ranked, cluster)
         : v == 2 ? fwd_cfg<768>(min_cls, ranked, cluster)
                  : fwd_cfg<1024>(min_cls, ranked, cluster);
}

cudaError_t launch_forward(const CallArgs& a, int variant, bool per_pair, cudaStream_t s) {
  if (!per_pair && a.cluster >= 2) {  // the cluster tier first: its pairs are the largest
    const cudaError_t e = variant == 1   ? launch_cluster<512>(a, s)
                          : variant == 2 ? launch_cluster<768>(a, s)
                                         : launch_cluster<1024>(a, s);
    if (e != cudaSuccess) return e;
  }
  return variant == 1   ? launch_fwd<512>(a, per_pair, s)
         : variant == 2 ? launch_fwd<768>(a, per_pair, s)
                        : launch_fwd<1024>(a, per_pair, s);
}

cudaError_t launch_match_deferred(const CallArgs& a, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int g = 4 * sm_count_of(dev);  // 32 warps per SM
  if (g <= 0) g = 4 * 152;
  if (a.P > 0) match_deferred_kernel<<<g, kDefNT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_match_only(const CallArgs& a, cudaStream_t s) {
  static DeviceOnce once;
  static int grid[kMaxDevices];
  const size_t sm = 2 * (3 * (size_t)kMaxBlocks + 16);
  int dev = 0;
  const cudaError_t e = once.run(
      [sm](int d) {
        grid[d] = sm_count_of(d);
        return cudaFuncSetAttribute(match_only_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      },
      &dev);
  if (e != cudaSuccess) return e;
  const int g = a.P < grid[dev] ? a.P : grid[dev];
  if (g > 0) match_only_kernel<<<g, kMatchNT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cfsim
