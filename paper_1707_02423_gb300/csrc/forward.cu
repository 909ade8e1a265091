// a2-a7: the batched similarity forward, greedy matching and graph score.
//
// One persistent kernel drains three cost-ordered queues (filled by plan.cu):
//   global class: pairs too large for shared memory; a CTA iterates X in a
//                 per-CTA scratch slot of the workspace (L2-resident),
//   CTA class:    a CTA keeps two iterates of X in shared memory,
//   warp class:   each warp keeps a small pair in its own shared-memory slice.
// Iteration (Table 1 "Iso" row, IsoRank-style, renormalised every step):
//   Y_{k+1} = alpha/2 (W_A X_k W_B^T + W_A^T X_k W_B) + (1 - alpha) Ehat,
//   X_{k+1} = Y_{k+1} / |Y_{k+1}|_F.
// The kernel stores Y (unnormalised) and carries s_k = 1/|Y_k|: because the
// propagation is linear, Z(X_k) = s_k Z(Y_k), so the norm is only needed
// after the gathers and each iteration has a single barrier (inside the
// fused Frobenius-norm reduction) with Y double-buffered.
//
// Thread mapping of a shared-memory pair (see Shape in layout.h): thread g
// owns column j = g % n_col of the resident matrix and rows r0 + R m.  The
// column graph's adjacency lists of j (first two entries, the common CFG
// degree) live in registers for the whole pair; the row graph's lists are
// read through the read-only cache and are uniform across the lanes that
// share a row.  Ehat of the owned entries stays in registers.
#include "device_common.cuh"
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
  const float* om;  // omega, shared-memory copy
  int F, Fp;
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
  g.s = classify(g.na, g.nb, cc);
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

// Adjacency lists of one column-graph block, first two entries in registers.
struct ColLists {
  int no, ni, vo0, vo1, vi0, vi1;
  float wo0, wo1, wi0, wi1;
  const CfAdj* po;
  const CfAdj* pi;
};

__device__ __forceinline__ ColLists load_col(const Geo& g, int j) {
  ColLists c;
  int e0 = __ldg(g.c_optr + j), e1 = __ldg(g.c_optr + j + 1);
  c.no = e1 - e0;
  c.po = g.c_oadj + e0;
  CfAdj x = c.no > 0 ? ldg_adj(c.po) : CfAdj{0, 0.f};
  c.vo0 = x.nbr;
  c.wo0 = x.w;
  x = c.no > 1 ? ldg_adj(c.po + 1) : CfAdj{0, 0.f};
  c.vo1 = x.nbr;
  c.wo1 = x.w;
  e0 = __ldg(g.c_iptr + j);
  e1 = __ldg(g.c_iptr + j + 1);
  c.ni = e1 - e0;
  c.pi = g.c_iadj + e0;
  x = c.ni > 0 ? ldg_adj(c.pi) : CfAdj{0, 0.f};
  c.vi0 = x.nbr;
  c.wi0 = x.w;
  x = c.ni > 1 ? ldg_adj(c.pi + 1) : CfAdj{0, 0.f};
  c.vi1 = x.nbr;
  c.wi1 = x.w;
  return c;
}

// sum over the column block's neighbours v of w_v * row[v]
__device__ __forceinline__ float dot_col(const float* row, int n, int v0, float w0, int v1, float w1,
                                        const CfAdj* p) {
  float t = 0.f;
  if (n > 0) t = w0 * row[v0];
  if (n > 1) t = fmaf(w1, row[v1], t);
  for (int f = 2; f < n; ++f) {
    CfAdj a = ldg_adj(p + f);
    t = fmaf(a.w, row[a.nbr], t);
  }
  return t;
}

// Successor-pair sum plus predecessor-pair sum for entry (i, j):
//   sum_{i->u} sum_{j->v} w_iu w_jv Y[u,v] + sum_{u->i} sum_{v->j} w_ui w_vj Y[u,v]
__device__ __forceinline__ float gather_s(const float* Y, int ld, const Geo& g, int i, const ColLists& c) {
  float s = 0.f;
  int e = __ldg(g.r_optr + i);
  const int e1 = __ldg(g.r_optr + i + 1);
  for (; e < e1; ++e) {
    const CfAdj a = ldg_adj(g.r_oadj + e);
    s = fmaf(a.w, dot_col(Y + a.nbr * ld, c.no, c.vo0, c.wo0, c.vo1, c.wo1, c.po), s);
  }
  int f = __ldg(g.r_iptr + i);
  const int f1 = __ldg(g.r_iptr + i + 1);
  for (; f < f1; ++f) {
    const CfAdj a = ldg_adj(g.r_iadj + f);
    s = fmaf(a.w, dot_col(Y + a.nbr * ld, c.ni, c.vi0, c.wi0, c.vi1, c.wi1, c.pi), s);
  }
  return s;
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

__device__ __forceinline__ float attr_norm(const float* a, const float* om, int F) {
  float acc = 0.f;
  for (int f = 0; f < F; ++f) {
    const float v = __ldg(a + f);
    acc = fmaf(om[f] * v, v, acc);
  }
  return sqrtf(acc);
}

__device__ __forceinline__ float attr_dot(const float* a, const float* b, const float* om, int F) {
  float acc = 0.f;
  for (int f = 0; f < F; ++f) acc = fmaf(om[f] * __ldg(a + f), __ldg(b + f), acc);
  return acc;
}

// a5-a6: greedy matching by rounds of locally dominant entries, and the score.
//
// Sequential greedy takes the largest remaining entry under the strict order
// (value desc, A index asc, B index asc).  An entry that is the largest of its
// row and of its column among the remaining rows/columns is taken by that
// greedy, so matching every such entry at once and repeating gives the same
// matching.  Within a row the order reduces to (value desc, column asc) and
// within a column to (value desc, row asc) in either orientation.
// State per row/column: >= 0 best live partner, -2 stale, -1 no candidate
// (only with NaN entries), <= -3 matched to (-3 - v).  Every round matches at
// least one pair for finite X, so the loop is bounded by min(n_row, n_col)
// rounds; if that bound is reached without a full matching (NaN in X) the
// status word gets CF_ERR_NUMERIC.  Returns the score on every thread; writes
// match[n_a] if given.
template <class Grp, class IdxT>
__device__ float greedy(const Grp grp, const float* X, int ld, int n_row, int n_col, int tr, IdxT* rb,
                        IdxT* nm, IdxT* cb, float* redf, int* redi, int32_t* mo, WsHeader* hdr, int pidx) {
  const int t = grp.rank(), G = Grp::size(), lane = t & 31, w = grp.warp(), NW = Grp::nwarps();
  for (int r = t; r < n_row; r += G) rb[r] = (IdxT)-2;
  for (int c = t; c < n_col; c += G) cb[c] = (IdxT)-2;
  grp.sync();
  const int need = min(n_row, n_col);
  int matched = 0, par = 0;
  for (int round = 0; matched < need && round < need; ++round) {
    for (int r = w; r < n_row; r += NW) {
      if (rb[r] != (IdxT)-2) continue;
      float bv = -CUDART_INF_F;
      int bi = 0x7fffffff;
      const float* xr = X + (size_t)r * ld;
      for (int c = lane; c < n_col; c += 32)
        if (cb[c] > (IdxT)-3) {
          const float v = xr[c];
          if (v > bv) {
            bv = v;
            bi = c;
          }
        }
      warp_argmax(bv, bi);
      if (lane == 0) rb[r] = bi == 0x7fffffff ? (IdxT)-1 : (IdxT)bi;
    }
    grp.sync();
    for (int c = w; c < n_col; c += NW) {
      if (cb[c] != (IdxT)-2) continue;
      float bv = -CUDART_INF_F;
      int bi = 0x7fffffff;
      for (int r = lane; r < n_row; r += 32)
        if (rb[r] > (IdxT)-3) {
          const float v = X[(size_t)r * ld + c];
          if (v > bv) {
            bv = v;
            bi = r;
          }
        }
      warp_argmax(bv, bi);
      if (lane == 0) cb[c] = bi == 0x7fffffff ? (IdxT)-1 : (IdxT)bi;
    }
    grp.sync();
    for (int r = t; r < n_row; r += G) {
      const int c = rb[r];
      nm[r] = (c >= 0 && cb[c] == r) ? (IdxT)c : (IdxT)-1;
    }
    grp.sync();
    int nn = 0;
    for (int r = t; r < n_row; r += G) {
      const int c = nm[r];
      if (c >= 0) {
        rb[r] = (IdxT)(-3 - c);
        cb[c] = (IdxT)(-3 - r);
        ++nn;
      }
    }
    matched += grp.sum_i(nn, redi, par);
    par ^= 1;
    for (int r = t; r < n_row; r += G) {
      const int c = rb[r];
      if (c >= 0 && cb[c] <= (IdxT)-3) rb[r] = (IdxT)-2;
    }
    grp.sync();
    for (int c = t; c < n_col; c += G) {
      const int r = cb[c];
      if (r >= 0 && rb[r] <= (IdxT)-3) cb[c] = (IdxT)-2;
    }
    grp.sync();
  }
  if (matched < need && grp.rank() == 0 && hdr) set_status(hdr, 6 /* CF_ERR_NUMERIC */, pidx);
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
  return grp.sum(sc, redf, 0);
}

// Write X_K (resident, possibly transposed, stride ld) to the caller's
// row-major n_a x n_b output, coalesced on the global side.
template <class Grp>
__device__ __forceinline__ void store_x(const Grp grp, const Ctx& cx, const Geo& g, const float* Xs, int ld) {
  float* dst = cx.X + cx.x_off[g.p];
  const int tot = g.na * g.nb;
  for (int idx = grp.rank(); idx < tot; idx += Grp::size()) {
    const int ia = idx / g.nb, jb = idx - ia * g.nb;
    const int r = g.s.tr ? jb : ia, c = g.s.tr ? ia : jb;
    dst[idx] = Xs[(size_t)r * ld + c];
  }
}

// A shared-memory-resident pair on a warp or a CTA.  buf0/buf1 hold the two
// iterates Y_k, Y_{k+1}; ehb holds (1 - alpha) Ehat.  Each thread reads and
// writes only its own entries of ehb, so ehb needs no barrier.
template <class Grp>
__device__ __forceinline__ void run_pair_s(const Ctx& cx, const Geo& g, const Grp grp, float* buf0, float* buf1,
                                           float* ehb, int16_t* ms, float* redf, int* redi) {
  const Shape& s = g.s;
  const int t = grp.rank();
  const bool act = t < s.R * s.n_col;
  const int j = act ? t % s.n_col : 0;
  const int r0 = act ? t / s.n_col : 0;
  const int Mt = (act && s.n_row > r0) ? ceil_div(s.n_row - r0, s.R) : 0;
  const int ld = s.ld;
  const int step = s.R * ld;
  const int off0 = r0 * ld + j;

  // a2: weighted attribute norms of the row blocks (buf1 is free until k = 0)
  for (int i = t; i < s.n_row; i += Grp::size()) buf1[i] = attr_norm(g.r_attr + (size_t)i * cx.Fp, cx.om, cx.F);
  const float* bcol = g.c_attr + (size_t)j * cx.Fp;
  const float cj = attr_norm(bcol, cx.om, cx.F);
  grp.sync();

  // a3: cosine attribute term E, its Frobenius norm, Ehat = X_0
  float ss = 0.f;
  for (int m = 0, i = r0, off = off0; m < Mt; ++m, i += s.R, off += step) {
    const float dot = attr_dot(g.r_attr + (size_t)i * cx.Fp, bcol, cx.om, cx.F);
    const float den = buf1[i] * cj;
    const float e = den > 0.f ? dot / den : 0.f;
    ehb[off] = e;
    ss = fmaf(e, e, ss);
  }
  const float tot = grp.sum(ss, redf, 0);
  const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  const float uni = 1.0f / sqrtf((float)s.n_row * (float)s.n_col);
  const float cb = 1.f - cx.alpha;
  for (int m = 0, off = off0; m < Mt; ++m, off += step) {
    const float eh = tot > 0.f ? ehb[off] * inv : uni;
    buf0[off] = eh;
    ehb[off] = cb * eh;
  }
  const ColLists cl = load_col(g, j);
  grp.sync();

  // a4: K renormalised iterations, one barrier each
  float sk = 1.f;
  for (int k = 0; k < cx.K; ++k) {
    const float* cur = (k & 1) ? buf1 : buf0;
    float* nxt = (k & 1) ? buf0 : buf1;
    const float ca = 0.5f * cx.alpha * sk;
    ss = 0.f;
    for (int m = 0, i = r0, off = off0; m < Mt; ++m, i += s.R, off += step) {
      const float y = fmaf(ca, gather_s(cur, ld, g, i, cl), ehb[off]);
      nxt[off] = y;
      ss = fmaf(y, y, ss);
    }
    const float yy = grp.sum(ss, redf, (k + 1) & 1);
    sk = cx.norm_mode == 0 ? 1.0f / sqrtf(yy) : 1.f;
  }
  float* Xs = (cx.K & 1) ? buf1 : buf0;
  if (sk != 1.f)
    for (int m = 0, off = off0; m < Mt; ++m, off += step) Xs[off] *= sk;
  grp.sync();

  if (cx.X) store_x(grp, cx, g, Xs, ld);
  if (cx.scores || cx.match) {
    int32_t* mo = cx.match ? cx.match + cx.m_off[g.p] : nullptr;
    const float sc = greedy<Grp, int16_t>(grp, Xs, ld, s.n_row, s.n_col, s.tr, ms, ms + s.n_row,
                                          ms + 2 * s.n_row, redf, redi, mo, cx.hdr, g.p);
    if (cx.scores && t == 0) cx.scores[g.p] = sc;
  }
  grp.sync();
}

// A global-class pair on a CTA: X, Ehat and the matching state in a scratch slot.
template <int NT>
__device__ void run_pair_g(const Ctx& cx, const Geo& g, float* slot, float* redf, int* redi) {
  const CtaGrp<NT> grp;
  const int n_row = g.na, n_col = g.nb;  // global-class shapes are never transposed
  const int64_t E = (int64_t)n_row * n_col;
  float* b0 = slot;
  float* b1 = b0 + E;
  float* eh = b1 + E;
  float* rn = eh + E;
  float* cn = rn + n_row;
  int32_t* ms = reinterpret_cast<int32_t*>(cn + n_col);
  const int t = threadIdx.x;
  for (int i = t; i < n_row; i += NT) rn[i] = attr_norm(g.r_attr + (size_t)i * cx.Fp, cx.om, cx.F);
  for (int jj = t; jj < n_col; jj += NT) cn[jj] = attr_norm(g.c_attr + (size_t)jj * cx.Fp, cx.om, cx.F);
  __syncthreads();
  float ss = 0.f;
  for (int64_t idx = t; idx < E; idx += NT) {
    const int i = (int)(idx / n_col), jj = (int)(idx - (int64_t)i * n_col);
    const float dot = attr_dot(g.r_attr + (size_t)i * cx.Fp, g.c_attr + (size_t)jj * cx.Fp, cx.om, cx.F);
    const float den = rn[i] * cn[jj];
    const float e = den > 0.f ? dot / den : 0.f;
    eh[idx] = e;
    ss = fmaf(e, e, ss);
  }
  const float tot = grp.sum(ss, redf, 0);
  const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  const float uni = 1.0f / sqrtf((float)n_row * (float)n_col);
  for (int64_t idx = t; idx < E; idx += NT) {
    const float v = tot > 0.f ? eh[idx] * inv : uni;
    eh[idx] = v;
    b0[idx] = v;
  }
  __syncthreads();
  float sk = 1.f;
  const float cbl = 1.f - cx.alpha;
  for (int k = 0; k < cx.K; ++k) {
    const float* cur = (k & 1) ? b1 : b0;
    float* nxt = (k & 1) ? b0 : b1;
    const float ca = 0.5f * cx.alpha * sk;
    ss = 0.f;
    for (int64_t idx = t; idx < E; idx += NT) {
      const int i = (int)(idx / n_col), jj = (int)(idx - (int64_t)i * n_col);
      const float y = fmaf(ca, gather_g(cur, n_col, g, i, jj), cbl * eh[idx]);
      nxt[idx] = y;
      ss = fmaf(y, y, ss);
    }
    const float yy = grp.sum(ss, redf, (k + 1) & 1);
    sk = cx.norm_mode == 0 ? 1.0f / sqrtf(yy) : 1.f;
  }
  float* Xs = (cx.K & 1) ? b1 : b0;
  if (sk != 1.f)
    for (int64_t idx = t; idx < E; idx += NT) Xs[idx] *= sk;
  __syncthreads();
  if (cx.X) store_x(grp, cx, g, Xs, n_col);
  if (cx.scores || cx.match) {
    int32_t* mo = cx.match ? cx.match + cx.m_off[g.p] : nullptr;
    const float sc = greedy<CtaGrp<NT>, int32_t>(grp, Xs, n_col, n_row, n_col, 0, ms, ms + n_row,
                                                 ms + 2 * n_row, redf, redi, mo, cx.hdr, g.p);
    if (cx.scores && t == 0) cx.scores[g.p] = sc;
  }
  __syncthreads();
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
    cx.pairs = a.pairs;
    cx.alpha = a.alpha;
    cx.K = a.K;
    cx.norm_mode = a.norm_mode;
    cx.X = a.X;
    cx.scores = a.scores;
    cx.match = a.match;
    cx.F = cx.A.F;
    cx.Fp = cx.A.F_pad;
    cx.om = s_om;
    *s_ok = (cx.A.F == cx.B.F && cx.A.F_pad == cx.B.F_pad) ? 1 : 0;
    if (!*s_ok && blockIdx.x == 0) set_status(cx.hdr, 1 /* CF_ERR_INVALID_ARG */, -1);
  }
  __syncthreads();
  if (!*s_ok) return false;
  if (threadIdx.x < kMaxF) {
    const float v = threadIdx.x < cx.F ? a.omega[threadIdx.x] : 0.f;
    s_om[threadIdx.x] = v;
    if (!(v >= 0.f && v <= 3.0e38f) && blockIdx.x == 0) set_status(cx.hdr, 6 /* CF_ERR_NUMERIC */, threadIdx.x);
  }
  __syncthreads();
  return true;
}

// Shared-memory layout of the batched kernel: three buffers of ccap floats
// (CTA class) which the warp class splits into NT/32 slices of three wcap
// buffers; then the larger of the CTA tail (reduction partials and int16
// matching state) and the warp tails (one matching state per warp).
__host__ __device__ constexpr size_t msw_bytes(int warp_rows) { return (2 * (2 * warp_rows + 48) + 15) / 16 * 16; }
__host__ __device__ constexpr size_t msc_bytes(int cta_rows, int nt) { return 512 + (2 * (2 * cta_rows + nt + 16) + 15) / 16 * 16; }
__host__ __device__ constexpr size_t fwd_smem_bytes(int nt, int ccap, int warp_rows, int cta_rows) {
  return 12 * (size_t)ccap + (msc_bytes(cta_rows, nt) > (size_t)(nt / 32) * msw_bytes(warp_rows)
                                  ? msc_bytes(cta_rows, nt)
                                  : (size_t)(nt / 32) * msw_bytes(warp_rows));
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fwd_batched_kernel(CallArgs a, ClassCfg cc, int per_pair) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_om[kMaxF];
  __shared__ uint32_t s_p;
  __shared__ Ctx s_cx;
  __shared__ int s_ok;
  if (!make_ctx(a, s_om, s_cx, &s_ok)) return;
  const Ctx& cx = s_cx;
  float* buf0 = reinterpret_cast<float*>(smem);
  float* buf1 = buf0 + cc.ccap;
  float* ehb = buf1 + cc.ccap;
  unsigned char* tail = smem + 12 * (size_t)cc.ccap;
  float* redf = reinterpret_cast<float*>(tail);
  int* redi = reinterpret_cast<int*>(tail + 256);
  int16_t* ms_c = reinterpret_cast<int16_t*>(tail + 512);
  const CtaGrp<NT> cta;

  if (per_pair >= 0) {  // the plain form: this launch runs exactly one pair on the CTA
    ClassCfg c1 = cc;
    c1.warp_rows = 0;  // no warp class: the whole CTA takes the pair
    const Geo g = make_geo(cx, per_pair, c1);
    if (g.s.cls == kClassGlobal) {
      const uint64_t need = global_slot_bytes(g.na, g.nb);
      if (need > cx.scratch_bytes) {
        if (threadIdx.x == 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, per_pair);
        return;
      }
      run_pair_g<NT>(cx, g, reinterpret_cast<float*>(cx.scratch), redf, redi);
    } else {
      run_pair_s<CtaGrp<NT>>(cx, g, cta, buf0, buf1, ehb, ms_c, redf, redi);
    }
    return;
  }

  const uint32_t nG = cx.hdr->n_class[kClassGlobal];
  const uint32_t nC = cx.hdr->n_class[kClassCta];
  const uint32_t nWp = cx.hdr->n_class[kClassWarp];
  // global class: one scratch slot per CTA
  if (nG > 0) {
    const uint64_t need = cx.hdr->slot_need;
    const uint64_t nslots = need ? cx.scratch_bytes / need : 0;
    if (nslots == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    } else if (blockIdx.x < nslots) {
      float* slot = reinterpret_cast<float*>(cx.scratch + (size_t)blockIdx.x * need);
      for (;;) {
        if (threadIdx.x == 0) s_p = atomicAdd(&cx.hdr->q_next[kClassGlobal], 1u);
        __syncthreads();
        const uint32_t q = s_p;
        __syncthreads();
        if (q >= nG) break;
        const Geo g = make_geo(cx, (int)cx.queue[q], cc);
        run_pair_g<NT>(cx, g, slot, redf, redi);
      }
    }
  }
  // CTA class
  for (;;) {
    if (threadIdx.x == 0) s_p = atomicAdd(&cx.hdr->q_next[kClassCta], 1u);
    __syncthreads();
    const uint32_t q = s_p;
    __syncthreads();
    if (q >= nC) break;
    const Geo g = make_geo(cx, (int)cx.queue[nG + q], cc);
    run_pair_s<CtaGrp<NT>>(cx, g, cta, buf0, buf1, ehb, ms_c, redf, redi);
  }
  // warp class: every warp drains the queue on its own slice
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpGrp wg{lane};
  float* wb0 = buf0 + (size_t)w * 3 * cc.wcap;
  float* wb1 = wb0 + cc.wcap;
  float* web = wb1 + cc.wcap;
  int16_t* ms_w = reinterpret_cast<int16_t*>(tail + (size_t)w * msw_bytes(cc.warp_rows));
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(&cx.hdr->q_next[kClassWarp], 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= nWp) break;
    const Geo g = make_geo(cx, (int)cx.queue[nG + nC + q], cc);
    run_pair_s<WarpGrp>(cx, g, wg, wb0, wb1, web, ms_w, nullptr, nullptr);
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
  const CtaGrp<kMatchNT> grp;
  for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
    const int pa = a.pairs[2 * p], pb = a.pairs[2 * p + 1];
    if (pa < 0 || pa >= A.n_cfgs || pb < 0 || pb >= B.n_cfgs) continue;  // recorded by the plan
    const int na = A.node_off[pa + 1] - A.node_off[pa];
    const int nb = B.node_off[pb + 1] - B.node_off[pb];
    const float* X = a.X_in + x_off[p];
    int32_t* mo = a.match ? a.match + m_off[p] : nullptr;
    const float sc = greedy<CtaGrp<kMatchNT>, int16_t>(grp, X, nb, na, nb, 0, ms, ms + na, ms + 2 * na, redf,
                                                       redi, mo, hdr, p);
    if (a.scores && threadIdx.x == 0) a.scores[p] = sc;
    __syncthreads();
  }
}

template <int NT, int MINB>
struct Variant {
  static cudaError_t launch(const CallArgs& a, const ClassCfg& cc, bool per_pair, cudaStream_t s) {
    static int blocks_per_sm = -1, n_sm = 0;
    const size_t sm = fwd_smem_bytes(NT, cc.ccap, cc.warp_rows, cc.cta_rows);
    if (blocks_per_sm < 0) {
      cudaError_t e =
          cudaFuncSetAttribute(fwd_batched_kernel<NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fwd_batched_kernel<NT, MINB>, NT, sm);
      if (e != cudaSuccess) return e;
      if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    if (per_pair) {
      for (int p = 0; p < a.P; ++p) fwd_batched_kernel<NT, MINB><<<1, NT, sm, s>>>(a, cc, p);
    } else {
      fwd_batched_kernel<NT, MINB><<<blocks_per_sm * n_sm, NT, sm, s>>>(a, cc, -1);
    }
    return cudaGetLastError();
  }
};

// 256 threads, three CTAs per SM: 3 x 5632 floats per CTA (66 KB) + tails.
constexpr ClassCfg kCfg0{256, 5632, 704, 256, 1024};
using V0 = Variant<256, 3>;

}  // namespace

int num_fwd_variants() { return 1; }

FwdVariant fwd_variant(int v) {
  (void)v;
  return FwdVariant{kCfg0.nt, 0, 3, kCfg0};
}

cudaError_t launch_forward(const CallArgs& a, int variant, bool per_pair, cudaStream_t s) {
  (void)variant;
  return V0::launch(a, kCfg0, per_pair, s);
}

cudaError_t launch_match_only(const CallArgs& a, cudaStream_t s) {
  static bool init = false;
  static int grid = 0;
  const size_t sm = 2 * (3 * (size_t)kMaxBlocks + 16);
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(match_only_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    grid = n_sm;
    init = true;
  }
  const int g = a.P < grid ? a.P : grid;
  if (g > 0) match_only_kernel<<<g, kMatchNT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cfsim
