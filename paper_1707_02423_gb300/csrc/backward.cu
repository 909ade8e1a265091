// a8: the adjoint of the similarity forward with the matching held fixed:
// gradients of sum_p g_p s_p with respect to every edge weight of both packs
// and to the per-feature attribute weights omega.
//
// Reverse mode of the forward (Table 1 "Cos" and "Iso" rows, renormalised):
//   Xbar_K   = g 1[matched entries]
//   for k = K-1 .. 0:
//     Ybar     = (Xbar - <Xbar, X_{k+1}> X_{k+1}) / |Y_{k+1}|   (Ybar = Xbar when not renormalised)
//     Ehatbar += (1 - alpha) Ybar ;  Zbar = alpha Ybar
//     Wbar_A  += 1/2 (Zbar W_B X_k^T + X_k W_B Zbar^T)  at A's edges
//     Wbar_B  += 1/2 (Zbar^T W_A X_k + X_k^T W_A Zbar)  at B's edges
//     Xbar     = 1/2 (W_A^T Zbar W_B + W_A Zbar W_B^T)   (the forward operator: it is self-adjoint)
//   Ehatbar += Xbar ;  Ebar = (Ehatbar - <Ehatbar, Ehat> Ehat) / |E|
//   omegabar_f = sum_ij Ebar_ij (a_if b_jf / (r_i c_j) - E_ij (a_if^2 / (2 r_i^2) + b_jf^2 / (2 c_j^2)))
// An edge p->q of A gets  1/2 sum over B's edges j->v of w_jv (Zbar[p,j] X_k[q,v] + X_k[p,j] Zbar[q,v]),
// and an edge j->v of B the same terms weighted by w_pq and summed over A's edges.
//
// X_k is needed in reverse order: the kernel first recomputes the forward,
// keeping X every S = ceil(sqrt(K)) steps and every |Y_k|, then walks the
// segments backwards, recomputing each segment's iterates from its checkpoint
// (about 2K forward steps and K adjoint steps; S + K/S + 1 matrices resident).
//
// A pair runs on a team: one 1024-thread CTA, or -- for the pairs too large
// for one CTA's shared memory in the forward, whose single-CTA adjoint would
// be the critical path of a batch -- all CTAs of a thread-block cluster.  All
// matrices live in a scratch slot of the workspace (L2-resident).  Element
// loops run a team warp per row and the lanes over columns.  An edge's
// gradient is a warp-reduced sum owned by one team warp per step,
// accumulated in the slot and added to a per-pack distinct-edge array when
// the pair is done; a last kernel adds those to the caller's user-order
// buffers.  Team syncs are CTA barriers or cluster barriers (release /
// acquire at cluster scope, which orders the slot's global-memory traffic).
#include "device_common.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

// A batch's adjoint time is the critical path of its largest pairs (a
// serial chain of about 3K sweeps, each ending in a team barrier), so teams
// are as wide as possible: 1024-thread CTAs (64 registers) beat 256- and
// 512-thread CTAs with more registers and more CTAs per SM (256 seeded
// pairs, n 10-300: 14.6 ms against 24.5 and 16.8 ms).
constexpr int kBwdNT = 1024;
constexpr int kBwdWarps = kBwdNT / 32;

// The threads working on one pair: one CTA (C == 1) or the C CTAs of a
// cluster.  Ranks and warps are numbered across the team.
struct Team {
  int rank, size, warp, nwarps, C;
  float* red;             // this CTA's per-warp partials, two parities
  float* part;            // this CTA's partial sums, two parities (cluster teams)
  const uint32_t* paddr;  // cluster address of every CTA's part[] (cluster teams)
  __device__ __forceinline__ void sync() const {
    if (C == 1)
      __syncthreads();
    else
      cl_sync();
  }
  // Sum over the team, the same bits on every thread.
  __device__ __forceinline__ float sum(float v, int par) const {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[par * 32 + w] = v;
    __syncthreads();
    const float cta = warp_sum(lane < kBwdWarps ? red[par * 32 + lane] : 0.f);
    if (C == 1) return cta;
    if (threadIdx.x == 0) part[par] = cta;
    cl_sync();
    return warp_sum(lane < C ? cl_ld_f32(paddr[lane] + 4u * par) : 0.f);
  }
};

struct BwdPair {
  int p, na, nb, ea, eb;
  const int32_t *ao, *ai, *bo, *bi;  // CFG-local row pointers (global edge indices)
  const CfAdj *aoa, *aia, *boa, *bia;
  const float *aat, *bat;  // attribute rows
  int a_edge0, b_edge0;    // first distinct edge of each CFG in its pack
};

struct BwdCtx {
  PackView A, B;
  const int32_t* pairs;
  const uint32_t* queue;
  const int64_t* m_off;
  const int32_t* match;
  const float* gbar;
  float* gcan_a;
  float* gcan_b;
  float* gomega;
  WsHeader* hdr;
  unsigned char* slots;
  size_t slots_bytes;
  const float* om;  // omega, shared-memory copy
  float alpha;
  int K, norm_mode, F, Fp;
  uint32_t n_pairs;  // valid pairs in the queue
};

// Successor-pair plus predecessor-pair sum of Y at entry (i, j) (A indexes
// rows, B columns; ld = n_b), both graphs' lists read from the pack.
__device__ __forceinline__ float gather_mem(const float* Y, const BwdPair& q, int i, int j) {
  float s = 0.f;
  const int c0 = q.bo[j], c1 = q.bo[j + 1];
  for (int e = q.ao[i], e1 = q.ao[i + 1]; e < e1; ++e) {
    const CfAdj a = q.aoa[e];
    const float* row = Y + (size_t)a.nbr * q.nb;
    float t = 0.f;
    for (int f = c0; f < c1; ++f) {
      const CfAdj b = q.boa[f];
      t = fmaf(b.w, row[b.nbr], t);
    }
    s = fmaf(a.w, t, s);
  }
  const int d0 = q.bi[j], d1 = q.bi[j + 1];
  for (int e = q.ai[i], e1 = q.ai[i + 1]; e < e1; ++e) {
    const CfAdj a = q.aia[e];
    const float* row = Y + (size_t)a.nbr * q.nb;
    float t = 0.f;
    for (int f = d0; f < d1; ++f) {
      const CfAdj b = q.bia[f];
      t = fmaf(b.w, row[b.nbr], t);
    }
    s = fmaf(a.w, t, s);
  }
  return s;
}

// One forward step with the normalisation carried, not applied: the stored
// iterates are Y_k (X_k = Y_k / |Y_k|), so from Y and inv = 1 / |Y| (1 for
// X_0 = Ehat, and always 1 when not renormalised) this writes
//   Yn = alpha/2 M(Y) inv + (1-alpha) Ehat
// and returns |Yn| (1 when not renormalised).  One pass, one team barrier.
__device__ __forceinline__ float fwd_step(const BwdCtx& cx, const BwdPair& q, const float* Y, float inv, float* Yn,
                                          const float* eh, const Team& tm, int& par) {
  const int lane = threadIdx.x & 31;
  const float ca = 0.5f * cx.alpha * inv, cb = 1.f - cx.alpha;
  float ss = 0.f;
  for (int i = tm.warp; i < q.na; i += tm.nwarps)
    for (int j = lane; j < q.nb; j += 32) {
      const size_t o = (size_t)i * q.nb + j;
      const float y = fmaf(ca, gather_mem(Y, q, i, j), cb * eh[o]);
      Yn[o] = y;
      ss = fmaf(y, y, ss);
    }
  const float yy = tm.sum(ss, par);
  par ^= 1;
  return cx.norm_mode != 0 ? 1.f : sqrtf(yy);
}

// Shared-memory accumulators of the B-edge gradients per CTA (floats): a
// pair whose B graph has more distinct edges uses a second sweep instead.
constexpr int kBwdEdgeAcc = 16384;

// gacc: this CTA's shared-memory accumulators of the B-edge gradients
// (kBwdEdgeAcc floats).
__device__ __forceinline__ void run_pair_bwd(const BwdCtx& cx, const BwdPair& q, float* slot, const Team& tm,
                                             float* gacc) {
  const int t = tm.rank, lane = threadIdx.x & 31, w = tm.warp;
  const int TN = tm.size, TW = tm.nwarps;
  const int na = q.na, nb = q.nb;
  const size_t E = (size_t)na * nb;
  const int K = cx.K, S = bwd_segment(K), nck = K / S + 1;
  // slot layout (bwd_slot_bytes)
  float* er = slot;                        // E (raw cosine term)
  float* eh = er + E;                      // Ehat
  float* ehb = eh + E;                     // Ehat-bar, then E-bar
  float* xb = ehb + E;                     // X-bar
  float* zb = xb + E;                      // Z-bar
  float* ck = zb + E;                      // checkpoints [nck][E]
  float* sg = ck + (size_t)nck * E;        // one segment's iterates [S + 1][E]
  float* nrm = sg + (size_t)(S + 1) * E;   // |Y_k|, k = 0..K
  float* rn = nrm + (K + 2);               // weighted attribute norms of A's blocks
  float* cn = rn + na;                     //   and of B's blocks
  float* rho = cn + nb;                    // sum_j Ebar_ij E_ij
  float* gam = rho + na;                   // sum_i Ebar_ij E_ij
  int* asrc = reinterpret_cast<int*>(gam + nb);
  int* adst = asrc + q.ea;
  float* aw = reinterpret_cast<float*>(adst + q.ea);
  float* ga = aw + q.ea;
  int* bsrc = reinterpret_cast<int*>(ga + q.ea);
  int* bdst = bsrc + q.eb;
  float* bw = reinterpret_cast<float*>(bdst + q.eb);
  float* gb = bw + q.eb;
  float* Rf = gb + q.eb;  // [na][Fp]: sum_j Ebar_ij b_jf / c_j
  int par = 0;
  float d_next = 0.f;  // <Xbar, X> of the adjoint step to come

  // both graphs' edge lists (CFG-local distinct-edge order), zeroed accumulators
  for (int i = t; i < na; i += TN)
    for (int e = __ldg(q.ao + i), e1 = __ldg(q.ao + i + 1); e < e1; ++e) {
      const CfAdj a = ldg_adj(q.aoa + e);
      const int l = e - q.a_edge0;
      asrc[l] = i;
      adst[l] = a.nbr;
      aw[l] = a.w;
      ga[l] = 0.f;
    }
  for (int j = t; j < nb; j += TN)
    for (int e = __ldg(q.bo + j), e1 = __ldg(q.bo + j + 1); e < e1; ++e) {
      const CfAdj b = ldg_adj(q.boa + e);
      const int l = e - q.b_edge0;
      bsrc[l] = j;
      bdst[l] = b.nbr;
      bw[l] = b.w;
      gb[l] = 0.f;
    }
  // E, |E|, Ehat = X_0 (checkpoint 0)
  for (int i = t; i < na; i += TN) rn[i] = attr_norm(q.aat + (size_t)i * cx.Fp, cx.om, cx.Fp);
  for (int j = t; j < nb; j += TN) cn[j] = attr_norm(q.bat + (size_t)j * cx.Fp, cx.om, cx.Fp);
  tm.sync();
  float ss = 0.f;
  for (int i = w; i < na; i += TW)
    for (int j = lane; j < nb; j += 32) {
      const float dot = attr_dot(q.aat + (size_t)i * cx.Fp, q.bat + (size_t)j * cx.Fp, cx.om, cx.Fp);
      const float den = rn[i] * cn[j];
      const float e = den > 0.f ? dot / den : 0.f;
      er[(size_t)i * nb + j] = e;
      ss = fmaf(e, e, ss);
    }
  const float nE = sqrtf(tm.sum(ss, par));
  par ^= 1;
  const float inv = nE > 0.f ? 1.f / nE : 0.f;
  const float uni = 1.f / sqrtf((float)na * (float)nb);
  for (int i = w; i < na; i += TW)
    for (int j = lane; j < nb; j += 32) {
      const size_t o = (size_t)i * nb + j;
      const float v = nE > 0.f ? er[o] * inv : uni;
      eh[o] = v;
      ck[o] = v;
    }
  if (t == 0) nrm[0] = 1.f;
  tm.sync();

  // forward, keeping Y every S steps (|Y_k| in nrm[k])
  {
    const float* Y = ck;
    float inv = 1.f;
    for (int k = 0; k < K; ++k) {
      float* dst = ((k + 1) % S == 0) ? ck + (size_t)((k + 1) / S) * E : sg + (size_t)((k + 1) % S) * E;
      const float nY = fwd_step(cx, q, Y, inv, dst, eh, tm, par);
      if (t == 0) nrm[k + 1] = nY;
      inv = 1.f / nY;
      Y = dst;
    }
    // Xbar_K = g 1[matched], Ehatbar = 0, and d = <Xbar_K, X_K> for the first adjoint step
    for (int i = w; i < na; i += TW)
      for (int j = lane; j < nb; j += 32) {
        const size_t o = (size_t)i * nb + j;
        xb[o] = 0.f;
        ehb[o] = 0.f;
      }
    tm.sync();
    const float g = cx.gbar[q.p];
    float acc = 0.f;
    for (int i = t; i < na; i += TN) {
      const int m = cx.match[cx.m_off[q.p] + i];
      if (m >= 0 && m < nb) {
        xb[(size_t)i * nb + m] = g;
        acc = fmaf(g, Y[(size_t)i * nb + m], acc);
      }
    }
    d_next = tm.sum(acc, par) * inv;  // also orders the xb writes
    par ^= 1;
  }
  // the B-edge gradient partials of this CTA (the edge loop computes each
  // (A edge, B edge) term once for both graphs' gradients)
  const bool eacc = q.eb <= kBwdEdgeAcc;
  if (eacc)
    for (int f = threadIdx.x; f < q.eb; f += kBwdNT) gacc[f] = 0.f;

  // adjoint sweep, one segment at a time from the last; two team barriers per step
  for (int seg = (K - 1) / S; seg >= 0 && K > 0; --seg) {
    const int k0 = seg * S, k1 = min(K, k0 + S);
    for (int i = w; i < na; i += TW)
      for (int j = lane; j < nb; j += 32) sg[(size_t)i * nb + j] = ck[(size_t)seg * E + (size_t)i * nb + j];
    tm.sync();
    for (int k = k0; k < k1 - 1; ++k)
      fwd_step(cx, q, sg + (size_t)(k - k0) * E, 1.f / nrm[k], sg + (size_t)(k - k0 + 1) * E, eh, tm, par);
    // the segment's last iterate Y_{k1} is the next checkpoint (or Y_K)
    const float* Yend = (k1 % S == 0) ? ck + (size_t)(k1 / S) * E : sg + (size_t)(k1 - k0) * E;
    if (k1 % S != 0) fwd_step(cx, q, sg + (size_t)(k1 - 1 - k0) * E, 1.f / nrm[k1 - 1], sg + (size_t)(k1 - k0) * E, eh, tm, par);
    for (int k = k1 - 1; k >= k0; --k) {
      const float* Y1 = (k + 1 == k1) ? Yend : sg + (size_t)(k + 1 - k0) * E;
      const float* Yk = sg + (size_t)(k - k0) * E;
      const bool nrmz = cx.norm_mode == 0;
      const float inv1 = nrmz ? 1.f / nrm[k + 1] : 1.f, invk = nrmz ? 1.f / nrm[k] : 1.f;
      // Ybar = (Xbar - <Xbar, X_{k+1}> X_{k+1}) / |Y_{k+1}|;  Ehatbar += (1-alpha) Ybar;  Zbar = alpha Ybar
      const float dd = nrmz ? d_next * inv1 : 0.f;
      for (int i = w; i < na; i += TW)
        for (int j = lane; j < nb; j += 32) {
          const size_t o = (size_t)i * nb + j;
          const float yb = (xb[o] - dd * Y1[o]) * inv1;
          ehb[o] = fmaf(1.f - cx.alpha, yb, ehb[o]);
          zb[o] = cx.alpha * yb;
        }
      tm.sync();
      // edge gradients at this step, from X_k = Yk invk
      for (int e = w; e < q.ea; e += TW) {
        const int p = asrc[e], qq = adst[e];
        const float we = aw[e] * invk;
        float s = 0.f;
        for (int f = lane; f < q.eb; f += 32) {
          const int j = bsrc[f], v = bdst[f];
          const float T = fmaf(zb[(size_t)p * nb + j], Yk[(size_t)qq * nb + v], Yk[(size_t)p * nb + j] * zb[(size_t)qq * nb + v]);
          s = fmaf(bw[f], T, s);
          if (eacc) atomicAdd(gacc + f, we * T);
        }
        s = warp_sum(s);
        if (lane == 0) ga[e] = fmaf(0.5f * invk, s, ga[e]);
      }
      if (!eacc)
        for (int f = w; f < q.eb; f += TW) {
          const int j = bsrc[f], v = bdst[f];
          float s = 0.f;
          for (int e = lane; e < q.ea; e += 32) {
            const int p = asrc[e], qq = adst[e];
            const float T = fmaf(zb[(size_t)p * nb + j], Yk[(size_t)qq * nb + v], Yk[(size_t)p * nb + j] * zb[(size_t)qq * nb + v]);
            s = fmaf(aw[e], T, s);
          }
          s = warp_sum(s);
          if (lane == 0) gb[f] = fmaf(0.5f * invk, s, gb[f]);
        }
      // Xbar_k = 1/2 M(Zbar), and <Xbar_k, X_k> for the next step
      float acc = 0.f;
      for (int i = w; i < na; i += TW)
        for (int j = lane; j < nb; j += 32) {
          const size_t o = (size_t)i * nb + j;
          const float x = 0.5f * gather_mem(zb, q, i, j);
          xb[o] = x;
          acc = fmaf(x, Yk[o], acc);
        }
      d_next = tm.sum(acc, par) * invk;  // a team barrier: Xbar_k complete
      par ^= 1;
    }
  }
  // Ehatbar += Xbar_0
  for (int i = w; i < na; i += TW)
    for (int j = lane; j < nb; j += 32) ehb[(size_t)i * nb + j] += xb[(size_t)i * nb + j];
  tm.sync();

  // omega gradient through the cosine term (rows / columns with a zero norm have E = 0 and no gradient)
  if (cx.gomega && nE > 0.f) {
    float acc = 0.f;
    for (int i = w; i < na; i += TW)
      for (int j = lane; j < nb; j += 32) acc = fmaf(ehb[(size_t)i * nb + j], eh[(size_t)i * nb + j], acc);
    const float d = tm.sum(acc, par);
    par ^= 1;
    for (int i = w; i < na; i += TW)
      for (int j = lane; j < nb; j += 32) {
        const size_t o = (size_t)i * nb + j;
        ehb[o] = (ehb[o] - d * eh[o]) / nE;  // Ebar
      }
    tm.sync();
    for (int i = w; i < na; i += TW) {
      float r = 0.f;
      for (int j = lane; j < nb; j += 32) r = fmaf(ehb[(size_t)i * nb + j], er[(size_t)i * nb + j], r);
      r = warp_sum(r);
      if (lane == 0) rho[i] = r;
      for (int f = 0; f < cx.F; ++f) {
        float s = 0.f;
        for (int j = lane; j < nb; j += 32)
          if (cn[j] > 0.f) s = fmaf(ehb[(size_t)i * nb + j], __ldg(q.bat + (size_t)j * cx.Fp + f) / cn[j], s);
        s = warp_sum(s);
        if (lane == 0) Rf[(size_t)i * cx.Fp + f] = s;
      }
    }
    for (int j = w; j < nb; j += TW) {
      float s = 0.f;
      for (int i = lane; i < na; i += 32) s = fmaf(ehb[(size_t)i * nb + j], er[(size_t)i * nb + j], s);
      s = warp_sum(s);
      if (lane == 0) gam[j] = s;
    }
    tm.sync();
    for (int f = w; f < cx.F; f += TW) {  // a warp per feature
      float g1 = 0.f, g2 = 0.f, g3 = 0.f;
      for (int i = lane; i < na; i += 32)
        if (rn[i] > 0.f) {
          const float a = __ldg(q.aat + (size_t)i * cx.Fp + f);
          g1 = fmaf(a / rn[i], Rf[(size_t)i * cx.Fp + f], g1);
          g2 = fmaf(a * a / (2.f * rn[i] * rn[i]), rho[i], g2);
        }
      for (int j = lane; j < nb; j += 32)
        if (cn[j] > 0.f) {
          const float b = __ldg(q.bat + (size_t)j * cx.Fp + f);
          g3 = fmaf(b * b / (2.f * cn[j] * cn[j]), gam[j], g3);
        }
      const float gsum = warp_sum(g1 - g2 - g3);
      if (lane == 0) atomicAdd(cx.gomega + f, gsum);
    }
  }
  // this pair's edge gradients into the packs' distinct-edge accumulators
  // (the B-edge sums from each CTA's shared-memory partials)
  for (int e = t; e < q.ea; e += TN) atomicAdd(cx.gcan_a + q.a_edge0 + e, ga[e]);
  if (eacc)
    for (int f = threadIdx.x; f < q.eb; f += kBwdNT) atomicAdd(cx.gcan_b + q.b_edge0 + f, 0.5f * gacc[f]);
  else
    for (int f = t; f < q.eb; f += TN) atomicAdd(cx.gcan_b + q.b_edge0 + f, gb[f]);
  tm.sync();
}

// Per-CTA setup by thread 0 into shared memory: pack views, workspace
// pointers, omega.
__device__ __forceinline__ void bwd_setup(const CallArgs& a, BwdCtx& c, float* s_om) {
  if (threadIdx.x == 0) {
    c.A = load_pack(a.pack_a);
    c.B = load_pack(a.pack_b);
    const WsLayout L = ws_layout(a.P);
    c.hdr = reinterpret_cast<WsHeader*>(a.ws + L.hdr);
    c.queue = reinterpret_cast<const uint32_t*>(a.ws + L.queue);
    c.m_off = reinterpret_cast<const int64_t*>(a.ws + L.m_off);
    const PackHeader* ha = reinterpret_cast<const PackHeader*>(a.pack_a);
    const PackHeader* hb = reinterpret_cast<const PackHeader*>(a.pack_b);
    const BwdLayout B = bwd_layout(a.P, ha->n_edges, hb->n_edges, a.pack_a == a.pack_b);
    c.gcan_a = reinterpret_cast<float*>(a.ws + B.grad_a);
    c.gcan_b = reinterpret_cast<float*>(a.ws + B.grad_b);
    c.slots = a.ws + B.slots;
    c.slots_bytes = a.ws_bytes > B.slots ? a.ws_bytes - B.slots : 0;
    c.pairs = a.pairs;
    c.match = a.match_in;
    c.gbar = a.grad_scores;
    c.gomega = a.grad_omega;
    c.alpha = a.alpha;
    c.K = a.K;
    c.norm_mode = a.norm_mode;
    c.F = c.A.F;
    c.Fp = c.A.F_pad;
    c.om = s_om;
    uint32_t n = 0;
    for (int k = 0; k < kNumClasses; ++k) n += c.hdr->n_class[k];
    c.n_pairs = n;
  }
  __syncthreads();
  if (threadIdx.x < kMaxF) s_om[threadIdx.x] = threadIdx.x < c.F ? a.omega[threadIdx.x] : 0.f;
  __syncthreads();
}

__device__ __forceinline__ BwdPair bwd_pair(const BwdCtx& cx, uint32_t qi) {
  BwdPair q;
  q.p = (int)cx.queue[qi];
  const int pa = cx.pairs[2 * q.p], pb = cx.pairs[2 * q.p + 1];
  const int ba = cx.A.node_off[pa], bb = cx.B.node_off[pb];
  q.na = cx.A.node_off[pa + 1] - ba;
  q.nb = cx.B.node_off[pb + 1] - bb;
  q.a_edge0 = cx.A.edge_off[pa];
  q.b_edge0 = cx.B.edge_off[pb];
  q.ea = cx.A.edge_off[pa + 1] - q.a_edge0;
  q.eb = cx.B.edge_off[pb + 1] - q.b_edge0;
  q.ao = cx.A.out_ptr + ba;
  q.ai = cx.A.in_ptr + ba;
  q.bo = cx.B.out_ptr + bb;
  q.bi = cx.B.in_ptr + bb;
  q.aoa = cx.A.out_adj;
  q.aia = cx.A.in_adj;
  q.boa = cx.B.out_adj;
  q.bia = cx.B.in_adj;
  q.aat = cx.A.attr + (size_t)ba * cx.Fp;
  q.bat = cx.B.attr + (size_t)bb * cx.Fp;
  return q;
}

// Pairs of at least this many entries take a whole cluster when clusters are
// launched (a pair's adjoint is a serial chain of sweeps over its entries,
// so the largest pairs need the widest teams); the others one CTA each.
constexpr int64_t kBwdBigEntries = 16384;

__device__ __forceinline__ bool bwd_big(const BwdPair& q) { return (int64_t)q.na * q.nb >= kBwdBigEntries; }

// One CTA per pair, every pair of the queue (used when no cluster of
// kBwdCluster CTAs fits on the device).
__global__ void __launch_bounds__(kBwdNT, 1) bwd_kernel(CallArgs a) {
  extern __shared__ __align__(16) float s_gacc[];  // kBwdEdgeAcc floats
  __shared__ __align__(16) float s_om[kMaxF];
  __shared__ float s_red[64];
  __shared__ BwdCtx s_cx;
  __shared__ uint32_t s_q;
  bwd_setup(a, s_cx, s_om);
  const BwdCtx& cx = s_cx;
  const uint64_t need = cx.hdr->bwd_slot_need;
  const uint64_t nslots = need ? cx.slots_bytes / need : 0;
  if (nslots == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && cx.n_pairs > 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    return;
  }
  if (blockIdx.x >= nslots) return;
  float* slot = reinterpret_cast<float*>(cx.slots + (size_t)blockIdx.x * need);
  const Team tm{(int)threadIdx.x, kBwdNT, (int)threadIdx.x >> 5, kBwdWarps, 1, s_red, nullptr, nullptr};
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(&cx.hdr->q_bwd, 1u);
    __syncthreads();
    const uint32_t qi = s_q;
    __syncthreads();
    if (qi >= cx.n_pairs) break;
    run_pair_bwd(cx, bwd_pair(cx, qi), slot, tm, s_gacc);
  }
}

// The whole batch on clusters of C CTAs.  First the large pairs (bwd_big,
// in queue order), each on a whole cluster: CTA 0 pulls a queue position and
// every CTA reads it through distributed shared memory, so all of them skip
// or take the same pairs; cluster c uses the scratch slot of its first CTA.
// Then every CTA on its own takes the other pairs with its own slot; a
// cluster's CTAs leave the first phase together (the pull that ends it is
// read between two cluster barriers), so no slot is used by two teams at
// once.  One kernel for both phases lets the small pairs fill SMs as soon as
// the large ones are done.
__global__ void __launch_bounds__(kBwdNT, 1) bwd_cluster_kernel(CallArgs a) {
  extern __shared__ __align__(16) float s_gacc[];  // kBwdEdgeAcc floats
  __shared__ __align__(16) float s_om[kMaxF];
  __shared__ float s_red[64];
  __shared__ float s_part[2];
  __shared__ uint32_t s_paddr[kMaxCluster];
  __shared__ BwdCtx s_cx;
  __shared__ uint32_t s_q, s_qaddr;
  bwd_setup(a, s_cx, s_om);
  const BwdCtx& cx = s_cx;
  const int C = (int)cl_size(), rank = (int)cl_rank();
  const uint32_t cid = cl_index();
  const uint64_t need = cx.hdr->bwd_slot_need;
  const uint64_t nslots = need ? cx.slots_bytes / need : 0;
  if (nslots == 0) {
    if (cid == 0 && rank == 0 && threadIdx.x == 0 && cx.n_pairs > 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    return;
  }
  if ((int)threadIdx.x < C) s_paddr[threadIdx.x] = cl_map(s_part, threadIdx.x);
  if (threadIdx.x == 0) s_qaddr = cl_map(&s_q, 0);
  __syncthreads();
  const uint64_t first_cta = (uint64_t)blockIdx.x - rank;  // the cluster's CTA 0
  if (first_cta < nslots) {  // the same on every CTA of the cluster
    float* slot = reinterpret_cast<float*>(cx.slots + first_cta * need);
    const Team tm{rank * kBwdNT + (int)threadIdx.x, C * kBwdNT, rank * kBwdWarps + ((int)threadIdx.x >> 5),
                  C * kBwdWarps, C, s_red, s_part, s_paddr};
    for (;;) {
      if (rank == 0 && threadIdx.x == 0) s_q = atomicAdd(&cx.hdr->q_bwd_big, 1u);
      cl_sync();
      const uint32_t qi = cl_ld_u32(s_qaddr);
      cl_sync();  // CTA 0 overwrites s_q only after every CTA has read it
      if (qi >= cx.n_pairs) break;
      const BwdPair q = bwd_pair(cx, qi);
      if (bwd_big(q)) run_pair_bwd(cx, q, slot, tm, s_gacc);
    }
  }
  if (blockIdx.x >= nslots) return;
  float* slot = reinterpret_cast<float*>(cx.slots + (uint64_t)blockIdx.x * need);
  const Team tm{(int)threadIdx.x, kBwdNT, (int)threadIdx.x >> 5, kBwdWarps, 1, s_red, nullptr, nullptr};
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(&cx.hdr->q_bwd, 1u);
    __syncthreads();
    const uint32_t qi = s_q;
    __syncthreads();
    if (qi >= cx.n_pairs) break;
    const BwdPair q = bwd_pair(cx, qi);
    if (!bwd_big(q)) run_pair_bwd(cx, q, slot, tm, s_gacc);
  }
}

// Zero the distinct-edge accumulators (sizes read from the pack headers).
__global__ void bwd_zero_kernel(CallArgs a) {
  const PackHeader* ha = reinterpret_cast<const PackHeader*>(a.pack_a);
  const PackHeader* hb = reinterpret_cast<const PackHeader*>(a.pack_b);
  const bool same = a.pack_a == a.pack_b;
  const BwdLayout B = bwd_layout(a.P, ha->n_edges, hb->n_edges, same);
  float* ga = reinterpret_cast<float*>(a.ws + B.grad_a);
  float* gb = reinterpret_cast<float*>(a.ws + B.grad_b);
  const int64_t n = ha->n_edges + (same ? 0 : hb->n_edges);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    (k < ha->n_edges ? ga[k] : gb[k - ha->n_edges]) = 0.f;
}

// out[e] += the distinct-edge gradient of user edge e, for every user edge.
__global__ void bwd_scatter_kernel(CallArgs a, int side) {
  const void* pack = side == 0 ? a.pack_a : a.pack_b;
  const PackHeader* ha = reinterpret_cast<const PackHeader*>(a.pack_a);
  const PackHeader* hb = reinterpret_cast<const PackHeader*>(a.pack_b);
  const BwdLayout B = bwd_layout(a.P, ha->n_edges, hb->n_edges, a.pack_a == a.pack_b);
  const float* g = reinterpret_cast<const float*>(a.ws + (side == 0 ? B.grad_a : B.grad_b));
  const PackView v = load_pack(pack);
  const int64_t n = reinterpret_cast<const PackHeader*>(pack)->n_user_edges;
  float* out = side == 0 ? a.grad_w_a : a.grad_w_b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] += g[v.u2c[e]];
}

int g_bwd_sm = 0;
int g_bwd_clusters = -1;  // resident clusters of kBwdCluster CTAs, 0 if none fit

constexpr int kBwdCluster = 8;
constexpr size_t kBwdSmem = sizeof(float) * kBwdEdgeAcc;

cudaLaunchConfig_t bwd_cluster_cfg(int n_clusters, cudaLaunchAttribute* attr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBwdCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(n_clusters * kBwdCluster, 1, 1);
  cfg.blockDim = dim3(kBwdNT, 1, 1);
  cfg.dynamicSmemBytes = kBwdSmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

cudaError_t launch_backward(const CallArgs& a, cudaStream_t s) {
  if (g_bwd_sm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&g_bwd_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  if (g_bwd_clusters < 0) {
    cudaError_t e = cudaFuncSetAttribute(bwd_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = bwd_cluster_cfg(1, attr, s);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, bwd_cluster_kernel, &cfg) != cudaSuccess) n = 0;
    cudaGetLastError();
    g_bwd_clusters = n;
  }
  bwd_zero_kernel<<<2 * g_bwd_sm, 256, 0, s>>>(a);
  if (g_bwd_clusters > 0) {  // large pairs on clusters, then the rest CTA by CTA, in one kernel
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = bwd_cluster_cfg(g_bwd_clusters, attr, s);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, bwd_cluster_kernel, a);
    if (e != cudaSuccess) return e;
  } else {  // no cluster fits: every pair on one CTA
    const int grid = a.P < 2 * g_bwd_sm ? a.P : 2 * g_bwd_sm;
    bwd_kernel<<<grid, kBwdNT, kBwdSmem, s>>>(a);
  }
  if (a.grad_w_a) bwd_scatter_kernel<<<2 * g_bwd_sm, 256, 0, s>>>(a, 0);
  if (a.grad_w_b && a.pack_a != a.pack_b) bwd_scatter_kernel<<<2 * g_bwd_sm, 256, 0, s>>>(a, 1);
  return cudaGetLastError();
}

}  // namespace cfsim
