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
// X_k is needed in reverse order: the forward is run once, keeping Y every
// S = ceil(sqrt(K)) steps (the checkpoints) and every 1/|Y_k|; the segments
// are then walked backwards, each recomputed from its checkpoint (the last one
// is still in place from the first pass), about 2K forward steps and K
// adjoint steps in all.
//
// Three tiers, by where a pair's matrices live (the forward's classes, sized
// for the adjoint's extra per-edge state):
//   resident (warp / eighth / quarter / half / whole CTA group): three
//     matrices in the group's shared-memory region -- the iterate being
//     gathered and the next one while the forward is recomputed; Y_k, Zbar
//     and Xbar during an adjoint step -- with the graphs staged as in the
//     forward.  Checkpoints, one segment of iterates, Ehat and the Ehat
//     adjoint sit in the group's slot of the workspace (L2-resident), read and
//     written entry by entry by each entry's owner (coalesced).
//   cluster: the same with the rows split over the CTAs of a thread-block
//     cluster (a slab each), gathers reading other CTAs' rows through
//     distributed shared memory, cluster barriers.
//   global: pairs too large for a cluster keep every matrix in an L2 slot
//     (one CTA or a whole cluster per pair, element loops over the slot).
// An adjoint step of a resident pair has two barriers: after the entrywise
// Ybar / Zbar pass (which also loads Y_k into shared memory), and inside the
// reduction of <Xbar_k, X_k> that ends the gather of Xbar_k and the edge
// terms.  Each (A edge, B edge) term is computed once for both graphs: a warp
// takes an edge of the row graph, its lanes the column graph's edges; the
// row edge's sum is a warp reduction, the column edges' sums shared-memory
// atomics.  A pair's edge sums go to per-pack distinct-edge accumulators when
// the pair is done; a last kernel adds those to the caller's user-order
// buffers.
#include <mutex>

#include "device_common.cuh"
#include "device_state.h"
#include "iterate.cuh"
#include "kernels.h"

namespace cfsim {

namespace {

// ---------------------------------------------------------------------------
// Global tier: every matrix of the pair in an L2 slot (bwd_slot_bytes layout).

// The threads working on one pair: one CTA (C == 1) or the C CTAs of a
// cluster.  Ranks and warps are numbered across the team.
struct Team {
  int rank, size, warp, nwarps, C, cta_warps;
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
    const float cta = warp_sum(lane < cta_warps ? red[par * 32 + lane] : 0.f);
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
  unsigned char* areas;  // per-CTA slot areas of the resident tier
  unsigned char* big;    // per-team slots of the cluster and global tiers
  size_t big_bytes;
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
__device__ __noinline__ void run_pair_bwd(const BwdCtx& cx, const BwdPair& q, float* slot, const Team& tm,
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
    for (int f = threadIdx.x; f < q.eb; f += blockDim.x) gacc[f] = 0.f;

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
    for (int f = threadIdx.x; f < q.eb; f += blockDim.x) atomicAdd(cx.gcan_b + q.b_edge0 + f, 0.5f * gacc[f]);
  else
    for (int f = t; f < q.eb; f += TN) atomicAdd(cx.gcan_b + q.b_edge0 + f, gb[f]);
  tm.sync();
}

// ---------------------------------------------------------------------------
// Resident tiers (groups of one CTA, and clusters).

// One pair oriented as the forward orients it: the row graph indexes the
// rows of the resident matrices (tr = 1 when that is B).
struct BGeo {
  Shape s;
  int p;
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

__device__ __forceinline__ BGeo make_bgeo(const BwdCtx& cx, int p, const ClassCfg& cc) {
  BGeo g;
  g.p = p;
  const int pa = __ldg(cx.pairs + 2 * p), pb = __ldg(cx.pairs + 2 * p + 1);
  const int ba = __ldg(cx.A.node_off + pa), bb = __ldg(cx.B.node_off + pb);
  const int na = __ldg(cx.A.node_off + pa + 1) - ba;
  const int nb = __ldg(cx.B.node_off + pb + 1) - bb;
  const int ea = __ldg(cx.A.edge_off + pa + 1) - __ldg(cx.A.edge_off + pa);
  const int eb = __ldg(cx.B.edge_off + pb + 1) - __ldg(cx.B.edge_off + pb);
  g.s = classify(na, nb, ea, eb, cc, __ldg(cx.A.xdeg + pa), __ldg(cx.B.xdeg + pb));
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

// The threads of a resident pair: a group of one CTA (kCl false), or the CTAs
// of a cluster, each thread of each CTA working on its CTA's slab of rows
// (kCl true; `cta` is then the whole CTA, used for CTA-local sums).
template <bool kCl>
struct RTeam {
  Group grp;     // the group (kCl false) or the whole CTA (kCl true)
  ClState* st;   // cluster state (kCl true)
  int C, rank;   // CTAs of the cluster and this CTA's rank (1, 0 for a group)
  __device__ __forceinline__ void sync() const {
    if (kCl)
      cl_sync();
    else
      grp.sync();
  }
  __device__ __forceinline__ float sum(float v, int par) const {
    if (kCl) return cl_sum(v, par, *st, C);
    return grp.sum(v, par);
  }
};

// Entry (i, j) of M(Y) for a staged row (A, Q, its ranges rr) and column (cl).
template <class YT>
__device__ __forceinline__ float gather_all(YT Y, const int4 A, const int4 Q, const int4* rr, int lr, const int2* redge,
                                            const int2* cedge, const int* cptr, const ColPad& cl, int n_col, int j) {
  float z = gather_fast(Y, A, Q, cl);
  if (A.w < 0 || cl.flag) {
    const int4 R4 = rr[lr];
    if (A.w < 0) z += row_extra(Y, R4, redge, cl);
    if (cl.flag) z += col_extra(Y, A, Q, R4, redge, cedge, cptr, n_col, j);
  }
  return z;
}

// M(buffer `b` of the three) at a staged entry: local shared loads, or -- in a
// cluster, for a row with a neighbour in another CTA (sign bit of A.y) --
// distributed-shared-memory loads relative to the owner's buffer 0.
template <bool kCl>
__device__ __forceinline__ float gather_buf(const float* buf, uint32_t boff, const int4 A, const int4 Q, const int4* rr,
                                            int lr, const int2* redge, const int2* cedge, const int* cptr,
                                            const ColPad& cl, int n_col, int j) {
  if (kCl && A.y < 0) return gather_all(ClusterY{boff}, A, Q, rr, lr, redge, cedge, cptr, cl, n_col, j);
  return gather_all(reinterpret_cast<const char*>(buf), A, Q, rr, lr, redge, cedge, cptr, cl, n_col, j);
}

__device__ __forceinline__ float lds_or_dsmem(const float* buf, uint32_t boff, int a, bool remote) {
  if (remote) return cl_ld_f32((uint32_t)a + boff);
  return *reinterpret_cast<const float*>(reinterpret_cast<const char*>(buf) + a);
}

// Entry loops over this thread's entries (offsets off0 + m step, m < Mt)
// that read one or two L2-resident slot matrices: the loads of eight entries
// are issued before any is used, so a loop waits for about one L2 round trip
// per eight entries instead of one per entry.
template <class F>
__device__ __forceinline__ void chunked1(int Mt, int off0, int step, const float* src, F&& f) {
  for (int m0 = 0; m0 < Mt; m0 += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (m0 + u < Mt) v[u] = __ldcg(src + off0 + (m0 + u) * step);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (m0 + u < Mt) f(off0 + (m0 + u) * step, v[u]);
  }
}
template <class F>
__device__ __forceinline__ void chunked2(int Mt, int off0, int step, const float* src0, const float* src1, F&& f) {
  for (int m0 = 0; m0 < Mt; m0 += 8) {
    float v[8], w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (m0 + u < Mt) {
        v[u] = __ldcg(src0 + off0 + (m0 + u) * step);
        w[u] = __ldcg(src1 + off0 + (m0 + u) * step);
      }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (m0 + u < Mt) f(off0 + (m0 + u) * step, v[u], w[u]);
  }
}

// This thread's view of a resident pair's staged lists and entries.
struct SweepGeo {
  const int4 *ra, *rq, *rr;
  const int2 *redge, *cedge;
  const int* cptr;
  const int16_t* brow;  // rows with further neighbours: (row, row mod R) pairs
  int nbr;              // their count
  int n_col, j, r0, Mt, R, ld, step, off0;
  ColPad cl;
};

// One sweep of M over this thread's entries:
//   out[off] = ca M(cur)[entry] + (base ? base[off] : 0),
// also stored to gdst[off] when given, and returns this thread's part of
// sum_entries out^2 (kDot false) or of sum_entries out[off] dotv[off] (kDot
// true).  In a group (kCl false) the main sweep is the straight-line 2 x 2
// gather for every entry with no branch; the terms of further neighbours are
// added afterwards -- a busy row's entries by their owners, a busy column's
// entries by the whole warp that holds the column (its owner's entries shared
// over the 32 lanes; the row fix-ups and a __syncwarp come first) -- so no
// lane's extra work stalls its warp.  Each entry is stored to gdst once, by
// whoever writes its final value.  In a cluster (kCl true) every entry takes
// its own further-neighbour terms, with distributed-shared-memory loads for
// rows that have a neighbour in another CTA.
template <bool kCl, bool kDot>
__device__ __forceinline__ float sweep(const SweepGeo& q, const float* cur, uint32_t boff, float ca, const float* base,
                                       float* out, float* gdst, const float* dotv) {
  float acc = 0.f;
#pragma unroll 2
  for (int m = 0; m < q.Mt; ++m) {
    const int lr = q.r0 + m * q.R, off = q.off0 + m * q.step;
    const int4 A = q.ra[lr], Q = q.rq[lr];
    float z;
    if (kCl)
      z = gather_buf<true>(cur, boff, A, Q, q.rr, lr, q.redge, q.cedge, q.cptr, q.cl, q.n_col, q.j);
    else
      z = gather_fast(reinterpret_cast<const char*>(cur), A, Q, q.cl);
    const float y = base ? fmaf(ca, z, base[off]) : ca * z;
    out[off] = y;
    if (gdst && (kCl || !(A.w < 0 || q.cl.flag))) gdst[off] = y;
    acc = kDot ? fmaf(y, dotv[off], acc) : fmaf(y, y, acc);
  }
  if (!kCl) {
    for (int b = 0; b < q.nbr; ++b) {
      if (q.Mt == 0 || q.brow[2 * b + 1] != q.r0) continue;  // a row of another thread
      const int i = q.brow[2 * b];
      const int off = i * q.ld + q.j;
      const float y0 = out[off];
      const float y = fmaf(ca, row_extra(reinterpret_cast<const char*>(cur), q.rr[i], q.redge, q.cl), y0);
      out[off] = y;
      if (gdst && !q.cl.flag) gdst[off] = y;
      acc += kDot ? (y - y0) * dotv[off] : y * y - y0 * y0;
    }
    __syncwarp();
    const int lane = threadIdx.x & 31;
    for (unsigned bm = __ballot_sync(0xffffffffu, q.cl.flag && q.Mt > 0); bm; bm &= bm - 1) {
      const int bl = __ffs(bm) - 1;
      const int jb = __shfl_sync(0xffffffffu, q.j, bl), ib = __shfl_sync(0xffffffffu, q.r0, bl);
      const int mb = __shfl_sync(0xffffffffu, q.Mt, bl);
      for (int m = lane; m < mb; m += 32) {
        const int i = ib + m * q.R, off = i * q.ld + jb;
        const float y0 = out[off];
        const float y = fmaf(ca,
                             col_extra(reinterpret_cast<const char*>(cur), q.ra[i], q.rq[i], q.rr[i], q.redge,
                                       q.cedge, q.cptr, q.n_col, jb),
                             y0);
        out[off] = y;
        if (gdst) gdst[off] = y;
        acc += kDot ? (y - y0) * dotv[off] : y * y - y0 * y0;
      }
    }
  }
  return acc;
}

// The adjoint of one resident pair.  For a group: all rows, region = the
// group's shared memory.  For a cluster: rows [i0, i0 + rows) of this CTA's
// slab; rbase[o] = cluster address of CTA o's region (zbytes long).  gslot:
// the pair's global slot (bwd_res_slot_bytes layout, full n_row x ld
// matrices).  When the region has room for a fourth matrix, the Ehat adjoint
// accumulates there instead of in the slot.
template <bool kCl>
__device__ __forceinline__ void run_pair_bwd_r(const BwdCtx& cx, const BGeo& g, const RTeam<kCl>& tm,
                                            unsigned char* region, size_t zbytes, float* gslot, size_t slot_bytes,
                                            const uint32_t* rbase) {
  const Shape& s = g.s;
  const int C = kCl ? tm.C : 1, crank = kCl ? tm.rank : 0;
  const int t = tm.grp.rank, G = tm.grp.size;
  const int lane = t & 31, wp = tm.grp.warp(), NW = tm.grp.nwarps();
  const int ld = s.ld, n_col = s.n_col;
  const int slab = kCl ? ceil_div(s.n_row, C) : s.n_row;
  const int i0 = crank * slab;
  const int rows = max(0, min(s.n_row, i0 + slab) - i0);
  const float gp = __ldg(cx.gbar + g.p);
  if (gp == 0.f) return;  // every term is linear in g: nothing to add (uniform over the team)
  const int ib = min(i0, s.n_row);  // a CTA past the last row has an empty slab
  const int eo0 = __ldg(g.r_optr), ei0 = __ldg(g.r_iptr);
  const int so0 = __ldg(g.r_optr + ib) - eo0, so1 = __ldg(g.r_optr + ib + rows) - eo0;
  const int si0 = __ldg(g.r_iptr + ib) - ei0, si1 = __ldg(g.r_iptr + ib + rows) - ei0;
  const int n_so = so1 - so0, n_si = si1 - si0;
  const int co0 = __ldg(g.c_optr), ci0 = __ldg(g.c_iptr);
  const int e_col = __ldg(g.c_optr + n_col) - co0;

  // ---- cluster: the halo.  The rows of other CTAs that this slab's rows
  // read are kept as extra rows of this CTA's own buffers (after its slab)
  // and copied from their owners once per sweep, so every gather and edge
  // term reads this CTA's shared memory.  Every CTA lays its buffers out for
  // the cluster's largest halo; a pair whose halo does not fit in some CTA's
  // region reads those rows through distributed shared memory instead.
  int H = 0, hmax = 0;
  bool halo = false;
  ClState* hs = tm.st;
  if (kCl) {
    const int nw = ceil_div(s.n_row, 32);
    const bool bitmap_ok = s.n_row <= kHaloMaxRows;
    for (int k = t; k < 64; k += G) hs->hbits[k] = 0u;
    __syncthreads();
    if (bitmap_ok)
      for (int lr = t; lr < rows; lr += G) {
        const int i = i0 + lr;
        for (int e = __ldg(g.r_optr + i) - eo0, e1 = __ldg(g.r_optr + i + 1) - eo0; e < e1; ++e) {
          const int u = __ldg(&g.r_oadj[eo0 + e].nbr);
          if ((u < i0 || u >= i0 + slab) && (unsigned)u < (unsigned)s.n_row) atomicOr(&hs->hbits[u >> 5], 1u << (u & 31));
        }
        for (int e = __ldg(g.r_iptr + i) - ei0, e1 = __ldg(g.r_iptr + i + 1) - ei0; e < e1; ++e) {
          const int u = __ldg(&g.r_iadj[ei0 + e].nbr);
          if ((u < i0 || u >= i0 + slab) && (unsigned)u < (unsigned)s.n_row) atomicOr(&hs->hbits[u >> 5], 1u << (u & 31));
        }
      }
    __syncthreads();
    if (t == 0) {
      int run = 0;
      for (int k = 0; k < nw && bitmap_ok; ++k) {
        hs->hpre[k] = run;
        run += __popc(hs->hbits[k]);
      }
      hs->hcnt = bitmap_ok && run <= kHaloRows ? run : (1 << 28);
    }
    __syncthreads();
    H = hs->hcnt;
    if (H <= kHaloRows)
      for (int u = t; u < s.n_row; u += G)
        if (hs->hbits[u >> 5] & (1u << (u & 31)))
          hs->hrow[hs->hpre[u >> 5] + __popc(hs->hbits[u >> 5] & ((1u << (u & 31)) - 1u))] = (int16_t)u;
    cl_sync();  // every CTA's count is published
    for (int o = 0; o < C; ++o) hmax = max(hmax, (int)cl_ld_u32(cl_map(&hs->hcnt, o)));
    // the layout this CTA would need with hmax halo rows per buffer
    const size_t nn_h = (size_t)(slab + hmax) * ld;
    const size_t end_h = align_up(12 * nn_h, 16) + 48 * (size_t)slab + 8 * (size_t)(n_so + n_si) + 16 * (size_t)e_col +
                         align_up(8 * (size_t)(n_col + 1), 16) + align_up(8 + 4 * (size_t)slab, 16) +
                         8 * (size_t)(n_so + e_col);
    if (t == 0) hs->hfit = hmax <= kHaloRows && end_h <= zbytes ? 1 : 0;
    cl_sync();
    halo = true;
    for (int o = 0; o < C; ++o) halo = halo && cl_ld_u32(cl_map(&hs->hfit, o)) != 0u;
  }
  const int nn = (slab + (halo ? hmax : 0)) * ld;
  float* B0 = reinterpret_cast<float*>(region);
  float* B1 = B0 + nn;
  float* B2 = B1 + nn;
  int4* ra = reinterpret_cast<int4*>(region + align_up(12 * (size_t)nn, 16));
  int4* rq = ra + slab;
  int4* rr = rq + slab;
  int2* redge = reinterpret_cast<int2*>(rr + slab);

  // ---- stage the lists (as the forward does), plus each edge's source and
  // a gradient accumulator per edge
  int2* cedge = redge + (n_so + n_si);
  int* cptr = reinterpret_cast<int*>(cedge + 2 * e_col);
  int* nbusy = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(cptr) + align_up(8 * (size_t)(n_col + 1), 16));
  int16_t* brow = reinterpret_cast<int16_t*>(nbusy + 2);  // [n_busy][2]: row, row mod R (groups only)
  int* rsrc = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(nbusy) + align_up(8 + 4 * (size_t)slab, 16));
  int* csrc = rsrc + n_so;
  float* gR = reinterpret_cast<float*>(csrc + e_col);
  float* gC = gR + n_so;
  float* B3 = reinterpret_cast<float*>(region + align_up((size_t)(reinterpret_cast<unsigned char*>(gC + e_col) - region), 16));
  const bool ehb_s = (size_t)(reinterpret_cast<unsigned char*>(B3) - region) + 4 * (size_t)nn <= zbytes;
  // (uniform over the team: every thread skips the pair together)
  if (!bounds_ok(cx.hdr, (size_t)(reinterpret_cast<unsigned char*>(gC + e_col) - region) <= zbytes, kSiteBwdRegion) ||
      !bounds_ok(cx.hdr, bwd_res_slot_bytes(s.n_row, ld, cx.K) <= slot_bytes, kSiteBwdSlot))
    return;
  const uint32_t buf_bytes = 4u * (uint32_t)nn;
  // row u as the gathers address it: a byte offset within this CTA's buffers
  // (a row of the slab, or a halo row after it), or -- a row with a
  // neighbour outside the slab, in a cluster without the halo -- the cluster
  // address of row u in its owner's buffer 0
  auto raddr = [&](int u, bool remote) -> int {
    if (kCl && halo && (u < i0 || u >= i0 + slab)) {
      const int h = hs->hpre[u >> 5] + __popc(hs->hbits[u >> 5] & ((1u << (u & 31)) - 1u));
      return (slab + h) * ld * 4;
    }
    if (!remote) return (u - i0) * ld * 4;
    const int o = u / slab;
    return (int)(rbase[o] + 4u * (uint32_t)((u - o * slab) * ld));
  };
  // copy this CTA's halo rows of a buffer (byte offset boff from buffer 0)
  // from their owners, then a CTA barrier; the owners' rows are final (a
  // cluster barrier came after they were written)
  auto pull = [&](float* buf, uint32_t boff) {
    for (int h = wp; h < H; h += NW) {
      const int u = hs->hrow[h];
      const int o = u / slab;
      const uint32_t src = rbase[o] + boff + 4u * (uint32_t)((u - o * slab) * ld);
      float* dst = buf + (size_t)(slab + h) * ld;
      for (int c0 = 0; c0 < n_col; c0 += 256) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + 32 * q + lane < n_col) v[q] = cl_ld_f32(src + 4u * (uint32_t)(c0 + 32 * q + lane));
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + 32 * q + lane < n_col) dst[c0 + 32 * q + lane] = v[q];
      }
    }
    __syncthreads();
  };
  for (int k = t; k < e_col; k += G) {
    CfAdj a = ldg_adj(g.c_oadj + co0 + k), b = ldg_adj(g.c_iadj + ci0 + k);
    if (!bounds_ok(cx.hdr, (unsigned)a.nbr < (unsigned)n_col && (unsigned)b.nbr < (unsigned)n_col, kSiteBwdColNbr))
      a.nbr = b.nbr = 0;
    cedge[k] = make_int2(4 * a.nbr, __float_as_int(a.w));
    cedge[e_col + k] = make_int2(4 * b.nbr, __float_as_int(b.w));
    gC[k] = 0.f;
  }
  for (int k = t; k <= n_col; k += G) {
    cptr[k] = __ldg(g.c_optr + k) - co0;
    cptr[n_col + 1 + k] = e_col + __ldg(g.c_iptr + k) - ci0;
  }
  for (int jj = t; jj < n_col; jj += G)
    for (int e = __ldg(g.c_optr + jj), e1 = __ldg(g.c_optr + jj + 1); e < e1; ++e) csrc[e - co0] = 4 * jj;
  for (int lr = t; lr < rows; lr += G) {
    const int i = i0 + lr;
    const int o0 = __ldg(g.r_optr + i) - eo0, o1 = __ldg(g.r_optr + i + 1) - eo0;
    const int q0 = __ldg(g.r_iptr + i) - ei0, q1 = __ldg(g.r_iptr + i + 1) - ei0;
    bool remote = false;
    if (kCl && !halo) {
      for (int e = o0; e < o1; ++e) {
        const int u = __ldg(&g.r_oadj[eo0 + e].nbr);
        remote |= u < i0 || u >= i0 + slab;
      }
      for (int e = q0; e < q1; ++e) {
        const int u = __ldg(&g.r_iadj[ei0 + e].nbr);
        remote |= u < i0 || u >= i0 + slab;
      }
    }
    const CfAdj z{i0, 0.f};  // padding: a valid row of this CTA, weight 0
    const CfAdj a0 = o1 > o0 ? ldg_adj(g.r_oadj + eo0 + o0) : z, a1 = o1 > o0 + 1 ? ldg_adj(g.r_oadj + eo0 + o0 + 1) : z;
    const CfAdj b0 = q1 > q0 ? ldg_adj(g.r_iadj + ei0 + q0) : z, b1 = q1 > q0 + 1 ? ldg_adj(g.r_iadj + ei0 + q0 + 1) : z;
    const int flag = (o1 - o0 > 2 || q1 - q0 > 2) ? (int)0x80000000 : 0;
    const int rflag = remote ? (int)0x80000000 : 0;
    ra[lr] = make_int4(raddr(a0.nbr, remote), __float_as_int(a0.w) | rflag, raddr(a1.nbr, remote),
                       __float_as_int(a1.w) | flag);
    rq[lr] = make_int4(raddr(b0.nbr, remote), __float_as_int(b0.w), raddr(b1.nbr, remote), __float_as_int(b1.w));
    rr[lr] = make_int4(o0 - so0, o1 - so0, n_so + q0 - si0, n_so + q1 - si0);
    for (int e = o0; e < o1; ++e) {
      CfAdj a = ldg_adj(g.r_oadj + eo0 + e);
      if (!bounds_ok(cx.hdr, (unsigned)a.nbr < (unsigned)s.n_row, kSiteBwdRowNbr)) a.nbr = i0;
      redge[e - so0] = make_int2(raddr(a.nbr, remote), __float_as_int(a.w));
      rsrc[e - so0] = (lr * ld * 4) | rflag;
      gR[e - so0] = 0.f;
    }
    for (int e = q0; e < q1; ++e) {
      CfAdj b = ldg_adj(g.r_iadj + ei0 + e);
      if (!bounds_ok(cx.hdr, (unsigned)b.nbr < (unsigned)s.n_row, kSiteBwdRowNbr)) b.nbr = i0;
      redge[n_so + e - si0] = make_int2(raddr(b.nbr, remote), __float_as_int(b.w));
    }
  }
  // this thread's entries: column j, local rows r0 + R m (m < Mt)
  const bool act = t < s.R * n_col;
  const int j = act ? t % n_col : 0;
  const int r0 = act ? t / n_col : 0;
  const int Mt = (act && rows > r0) ? ceil_div(rows - r0, s.R) : 0;
  const int step = s.R * ld;
  const int off0 = r0 * ld + j;
  const size_t gbase = (size_t)i0 * ld;  // global offset of this CTA's first row
  // the pair's global slot
  const int K = cx.K, S = bwd_segment(K), nck = K / S + 1;
  const size_t NE = (size_t)s.n_row * ld;
  float* ginv = gslot;  // 1 / |Y_k| (1 when not renormalised), k = 0..K
  float* mats = gslot + bwd_res_norm_floats(K);
  float* g_eh = mats + (size_t)(nck + S) * NE;
  float* g_ehb = g_eh + NE;
  float* g_xbs = g_ehb + NE;
  auto yloc = [&](int k) -> float* { return mats + (size_t)(k % S == 0 ? k / S : nck + k % S) * NE; };
  const bool nrmz = cx.norm_mode == 0;
  const float alpha = cx.alpha, cb = 1.f - alpha;
  int par = 0;

  // ---- a3: E, |E|, Ehat = X_0 (row norms staged in B1, this column's in a register)
  for (int lr = t; lr < rows; lr += G) B1[lr] = attr_norm(g.r_attr + (size_t)(i0 + lr) * cx.Fp, cx.om, cx.Fp);
  const float* bcol = g.c_attr + (size_t)j * cx.Fp;
  const float cj = attr_norm(bcol, cx.om, cx.Fp);
  tm.sync();
  float ss = 0.f;
  for (int m = 0, lr = r0, off = off0; m < Mt; ++m, lr += s.R, off += step) {
    const float dot = attr_dot(g.r_attr + (size_t)(i0 + lr) * cx.Fp, bcol, cx.om, cx.Fp);
    const float den = B1[lr] * cj;
    const float e = den > 0.f ? dot / den : 0.f;
    B0[off] = e;
    ss = fmaf(e, e, ss);
  }
  const float tot = tm.sum(ss, par);  // also: every read of B1 is done
  par ^= 1;
  const float nE = sqrtf(tot);
  const float einv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  const float uni = 1.0f / sqrtf((float)s.n_row * (float)n_col);
  for (int m = 0, off = off0; m < Mt; ++m, off += step) {
    const float eh = tot > 0.f ? B0[off] * einv : uni;
    B0[off] = eh;
    B2[off] = cb * eh;
    g_eh[gbase + off] = eh;
    mats[gbase + off] = eh;  // checkpoint 0
  }
  if (t == 0) ginv[0] = 1.f;
  tm.sync();  // Y_0 and the staged lists visible
  if (!kCl && wp == 0) {  // the rows with further neighbours, in index order (warp 0 of the group)
    int cnt = 0;
    for (int b = 0; b < rows; b += 32) {
      const int i = b + lane;
      const bool x = i < rows && ra[i].w < 0;
      const unsigned msk = __ballot_sync(0xffffffffu, x);
      if (x) {
        const int qq = cnt + __popc(msk & ((1u << lane) - 1u));
        brow[2 * qq] = (int16_t)i;
        brow[2 * qq + 1] = (int16_t)(i % s.R);
      }
      cnt += __popc(msk);
    }
    if (lane == 0) *nbusy = cnt;
  }
  tm.grp.sync();
  SweepGeo sq;
  sq.ra = ra;
  sq.rq = rq;
  sq.rr = rr;
  sq.redge = redge;
  sq.cedge = cedge;
  sq.cptr = cptr;
  sq.brow = brow;
  sq.nbr = kCl ? 0 : *nbusy;
  sq.n_col = n_col;
  sq.j = j;
  sq.r0 = r0;
  sq.Mt = Mt;
  sq.R = s.R;
  sq.ld = ld;
  sq.step = step;
  sq.off0 = off0;
  sq.cl = load_col(cptr, cedge, n_col, j);

  // ---- the forward, once: Y_k to its place in the slot, 1/|Y_k| to ginv
  float sk = 1.f;
  for (int k = 0; k < K; ++k) {
    const float* cur = (k & 1) ? B1 : B0;
    float* nxt = (k & 1) ? B0 : B1;
    float* dst = yloc(k + 1) + gbase;
    const float ca = 0.5f * alpha * sk;
    if (kCl && halo) pull(const_cast<float*>(cur), (k & 1) ? buf_bytes : 0u);
    ss = sweep<kCl, false>(sq, cur, (k & 1) ? buf_bytes : 0u, ca, B2, nxt, dst, nullptr);
    const float yy = tm.sum(ss, par);
    par ^= 1;
    sk = nrmz ? 1.0f / sqrtf(yy) : 1.f;
    if (t == 0) ginv[k + 1] = sk;
  }

  // ---- Xbar_K = g 1[matched] (in B2) and d = <Xbar_K, X_K>
  const float* YK = (K & 1) ? B1 : B0;
  const int64_t mo = cx.m_off[g.p];
  const int mcol = s.tr ? cx.match[mo + j] : -1;  // A block = this column: its matched B block (a row)
  float acc = 0.f;
  for (int m = 0, lr = r0, off = off0; m < Mt; ++m, lr += s.R, off += step) {
    const bool hit = s.tr ? (mcol == i0 + lr) : (cx.match[mo + i0 + lr] == j);
    const float xb = hit ? gp : 0.f;
    B2[off] = xb;
    if (ehb_s)
      B3[off] = 0.f;
    else
      g_ehb[gbase + off] = 0.f;
    acc = fmaf(xb, YK[off], acc);
  }
  float d = tm.sum(acc, par) * sk;
  par ^= 1;

  // ---- the adjoint, segment by segment from the last (which is in place)
  const int nseg = K > 0 ? (K - 1) / S + 1 : 0;
  float* XB = B2;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * S, k1 = min(K, k0 + S);
    const bool last = seg == nseg - 1;
    float* XK = last ? ((K & 1) ? B1 : B0) : B0;
    float* ZB = last ? ((K & 1) ? B0 : B1) : B1;
    if (!last) {
      // stash Xbar_{k1}; recompute Y_{k0+1} .. Y_{k1-1} from checkpoint seg
      const float* ck = mats + (size_t)seg * NE + gbase;
      chunked2(Mt, off0, step, g_eh + gbase, ck, [&](int off, float eh, float y0) {
        g_xbs[gbase + off] = B2[off];
        B2[off] = cb * eh;
        B0[off] = y0;
      });
      tm.sync();
      for (int k = k0; k < k1 - 1; ++k) {
        const int u = k - k0;
        const float* cur = (u & 1) ? B1 : B0;
        float* nxt = (u & 1) ? B0 : B1;
        float* dst = yloc(k + 1) + gbase;
        const float ca = 0.5f * alpha * ginv[k];
        if (kCl && halo) pull(const_cast<float*>(cur), (u & 1) ? buf_bytes : 0u);
        sweep<kCl, false>(sq, cur, (u & 1) ? buf_bytes : 0u, ca, B2, nxt, dst, nullptr);
        tm.sync();
      }
      chunked1(Mt, off0, step, g_xbs + gbase, [&](int off, float x) { B2[off] = x; });
    }
    const uint32_t zoff = ZB == B0 ? 0u : buf_bytes;   // byte offset of ZB from buffer 0
    const uint32_t xoff = XK == B0 ? 0u : buf_bytes;
    for (int k = k1 - 1; k >= k0; --k) {
      const float inv1 = ginv[k + 1], invk = ginv[k];
      const float dd = nrmz ? d * inv1 : 0.f;
      const float* y1g = (k == k1 - 1 && !last) ? yloc(k1) + gbase : nullptr;
      const float* ykg = yloc(k) + gbase;
      // entrywise: Ybar, Ehatbar += (1-alpha) Ybar, Zbar = alpha Ybar; Y_k into XK
      chunked1(Mt, off0, step, ykg, [&](int off, float yk) {
        const float y1 = y1g ? y1g[off] : XK[off];
        const float yb = (XB[off] - dd * y1) * inv1;
        if (ehb_s)
          B3[off] = fmaf(cb, yb, B3[off]);
        else
          atomicAdd(g_ehb + gbase + off, cb * yb);  // a reduction at L2: nothing waits for it
        ZB[off] = alpha * yb;
        XK[off] = yk;
      });
      tm.sync();
      // Xbar_k = 1/2 M(Zbar) and <Xbar_k, Y_k>
      if (kCl && halo) {
        pull(ZB, zoff);
        pull(XK, xoff);
      }
      acc = sweep<kCl, true>(sq, ZB, zoff, 0.5f, nullptr, XB, nullptr, XK);
      // edge terms T = Zbar[p,j] Y_k[q,v] + Y_k[p,j] Zbar[q,v] for row edge p->q, column edge j->v:
      // lanes take the column edges 32 at a time, warps the row edges; a row
      // edge's sum is a warp reduction, a column edge's sum over this warp's
      // row edges one shared-memory atomic per lane and chunk
      const float hinv = 0.5f * invk;
      for (int c0 = 0; c0 < e_col; c0 += 32) {
        const int f = c0 + lane;
        const bool fv = f < e_col;
        const int2 ce = fv ? cedge[f] : make_int2(0, 0);
        const int cs = fv ? csrc[f] : 0;
        const float wf = __int_as_float(ce.y);  // 0 for lanes past the end
        float cacc = 0.f;
        for (int e = wp; e < n_so; e += NW) {
          const int rs = rsrc[e];
          const int2 re = redge[e];
          const bool rem = kCl && rs < 0;
          const int a1 = (rs & 0x7fffffff) + cs, a2 = re.x + ce.x;
          const float z1 = *reinterpret_cast<const float*>(reinterpret_cast<const char*>(ZB) + a1);
          const float x1 = *reinterpret_cast<const float*>(reinterpret_cast<const char*>(XK) + a1);
          const float z2 = lds_or_dsmem(ZB, zoff, a2, rem), x2 = lds_or_dsmem(XK, xoff, a2, rem);
          const float T = fmaf(z1, x2, x1 * z2);
          cacc = fmaf(__int_as_float(re.y), T, cacc);
          const float sr = warp_sum(wf * T);
          if (lane == 0) gR[e] = fmaf(hinv, sr, gR[e]);
        }
        if (fv && cacc != 0.f) atomicAdd(gC + f, hinv * cacc);
      }
      d = tm.sum(acc, par) * invk;  // barrier: Xbar_k, the edge terms and every read of ZB / XK done
      par ^= 1;
    }
  }

  // ---- Ehatbar += Xbar_0 (into the slot), then the omega gradient through the cosine term
  if (ehb_s) {
    for (int m = 0, off = off0; m < Mt; ++m, off += step) g_ehb[gbase + off] = B3[off] + XB[off];
  } else {
    __threadfence();  // this thread's reductions into its entries are performed before it reads them
    chunked1(Mt, off0, step, g_ehb + gbase, [&](int off, float e) { g_ehb[gbase + off] = e + XB[off]; });
  }
  if (cx.gomega && nE > 0.f) {
    acc = 0.f;
    chunked2(Mt, off0, step, g_ehb + gbase, g_eh + gbase, [&](int, float e, float h) { acc = fmaf(e, h, acc); });
    const float dot = tm.sum(acc, par);  // also orders every B0 / B1 read above before the staging below
    par ^= 1;
    // 1 / r_i of this CTA's rows and 1 / c_j of the columns (0 for a zero norm)
    for (int lr = t; lr < rows; lr += G) {
      const float r = attr_norm(g.r_attr + (size_t)(i0 + lr) * cx.Fp, cx.om, cx.Fp);
      B0[lr] = r > 0.f ? 1.f / r : 0.f;
    }
    for (int jj = t; jj < n_col; jj += G) {
      const float c = attr_norm(g.c_attr + (size_t)jj * cx.Fp, cx.om, cx.Fp);
      B1[jj] = c > 0.f ? 1.f / c : 0.f;
    }
    tm.sync();
    const float cinv = B1[j];
    const float einv_n = 1.f / nE;
    for (int q = 0; q < (cx.Fp >> 2); ++q) {
      float4 gacc = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 b4 = __ldg(reinterpret_cast<const float4*>(bcol) + q);
      const float4 bt = make_float4(b4.x * cinv, b4.y * cinv, b4.z * cinv, b4.w * cinv);
      for (int m = 0, lr = r0, off = off0; m < Mt; ++m, lr += s.R, off += step) {
        const float eh = __ldcg(g_eh + gbase + off);
        const float ebar = (__ldcg(g_ehb + gbase + off) - dot * eh) * einv_n;  // Ebar
        const float E = eh * nE;
        const float ri = B0[lr];
        const float4 a4 = __ldg(reinterpret_cast<const float4*>(g.r_attr + (size_t)(i0 + lr) * cx.Fp) + q);
        const float4 at = make_float4(a4.x * ri, a4.y * ri, a4.z * ri, a4.w * ri);
        gacc.x = fmaf(ebar, fmaf(-0.5f * E, fmaf(at.x, at.x, bt.x * bt.x), at.x * bt.x), gacc.x);
        gacc.y = fmaf(ebar, fmaf(-0.5f * E, fmaf(at.y, at.y, bt.y * bt.y), at.y * bt.y), gacc.y);
        gacc.z = fmaf(ebar, fmaf(-0.5f * E, fmaf(at.z, at.z, bt.z * bt.z), at.z * bt.z), gacc.z);
        gacc.w = fmaf(ebar, fmaf(-0.5f * E, fmaf(at.w, at.w, bt.w * bt.w), at.w * bt.w), gacc.w);
      }
      // this CTA part's sums (no cluster barrier: each CTA adds its own)
      const float g0 = tm.grp.sum(gacc.x, par);
      const float g1 = tm.grp.sum(gacc.y, par ^ 1);
      const float g2 = tm.grp.sum(gacc.z, par);
      const float g3 = tm.grp.sum(gacc.w, par ^ 1);
      if (t == 0) {
        if (4 * q + 0 < cx.F) atomicAdd(cx.gomega + 4 * q + 0, g0);
        if (4 * q + 1 < cx.F) atomicAdd(cx.gomega + 4 * q + 1, g1);
        if (4 * q + 2 < cx.F) atomicAdd(cx.gomega + 4 * q + 2, g2);
        if (4 * q + 3 < cx.F) atomicAdd(cx.gomega + 4 * q + 3, g3);
      }
    }
  }
  // ---- this pair's edge gradients into the packs' distinct-edge accumulators
  tm.grp.sync();  // this CTA's gR / gC complete
  float* gcR = s.tr ? cx.gcan_b : cx.gcan_a;
  float* gcC = s.tr ? cx.gcan_a : cx.gcan_b;
  for (int e = t; e < n_so; e += G) atomicAdd(gcR + eo0 + so0 + e, gR[e]);
  for (int f = t; f < e_col; f += G) atomicAdd(gcC + co0 + f, gC[f]);
  tm.sync();  // the region and the slot are free for the next pair (cluster: every CTA done reading remote rows)
}

// Per-CTA setup by thread 0 into shared memory: pack views, workspace
// pointers, omega.
__device__ __forceinline__ void bwd_setup(const CallArgs& a, BwdCtx& c, float* s_om, int n_cta, size_t area) {
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
    c.areas = a.ws + B.slots;
    const size_t big0 = B.slots + (size_t)n_cta * area;
    c.big = a.ws + big0;
    c.big_bytes = a.ws_bytes > big0 ? a.ws_bytes - big0 : 0;
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

__device__ __forceinline__ BwdPair bwd_pair(const BwdCtx& cx, int p) {
  BwdPair q;
  q.p = p;
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

// Shape of the adjoint kernel: the forward's group levels and regions, sized
// for the adjoint (ClassCfg::bwd).
constexpr size_t kBwdSmem = 225280;
template <int NT>
__host__ __device__ constexpr ClassCfg bwd_cfg(int cluster) {
  return ClassCfg{NT,
                  (int)kBwdSmem,
                  (int)kBwdSmem / 2,
                  (int)kBwdSmem / 4,
                  (int)kBwdSmem / 8,
                  ((int)kBwdSmem / (NT / 32)) & ~15,
                  kClassWarp,
                  0,
                  cluster,
                  1};
}

// Bytes of one CTA's slot area: the slots of its groups at every level, each
// at its region's offset scaled by bwd_slot_ratio_q.
template <int NT>
__host__ __device__ size_t bwd_area_bytes(int K) {
  const uint64_t q = bwd_slot_ratio_q(K, (size_t)bwd_cfg<NT>(0).z_wrp);
  return bwd_slot_at(kBwdSmem, q) + kAlign;
}

// The adjoint's per-CTA shared state and setup of both kernels.
template <int NT>
struct BwdShared {
  float om[kMaxF];
  BwdCtx cx;
  ClState st;
  uint32_t p[1 + 2 + 4 + 8 + NT / 32];  // queue positions: CTA, half, quarter, eighth groups, warps
  float redf[4][2 * NT / 32];
  int redi[4][2 * NT / 32];
};

// The pairs that fit no single CTA, each on a whole team: a cluster of C CTAs
// (launched as clusters) or one CTA (C = 1).  First the global class out of
// an L2 slot, then the cluster class resident in the cluster's shared memory.
// CTA 0 of a cluster pulls a queue position and every CTA reads it through
// distributed shared memory, so all of them take the same pairs.  Team c uses
// slot c of the team slots.
template <int NT>
__global__ void __launch_bounds__(NT, 1) bwd_big_kernel(CallArgs a, int n_cta) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) BwdShared<NT> sh;
  bwd_setup(a, sh.cx, sh.om, n_cta, bwd_area_bytes<NT>(a.K));
  const BwdCtx& cx = sh.cx;
  ClState& st = sh.st;
  const int t = threadIdx.x;
  const int C = (int)cl_size(), rank = (int)cl_rank();
  const uint32_t cid = C > 1 ? cl_index() : blockIdx.x;
  const ClassCfg cc = bwd_cfg<NT>(C > 1 ? C : 0);
  const uint32_t n_gl = cx.hdr->n_class[kClassGlobal], n_cl = cx.hdr->n_class[kClassCluster];
  if (n_gl + n_cl == 0) return;
  const uint64_t need = cx.hdr->bwd_big_need;
  const uint64_t nslots = need ? cx.big_bytes / need : 0;
  if (nslots == 0) {
    if (blockIdx.x == 0 && t == 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    return;
  }
  if (cid >= nslots) return;  // the same on every CTA of a cluster
  if (t < C) {
    st.rbase[t] = cl_map(smem, t);
    st.paddr[t] = cl_map(st.part, t);
    st.piaddr[t] = cl_map(st.parti, t);
  }
  if (t == 0) st.qaddr = cl_map(&st.q, 0);
  __syncthreads();
  unsigned char* slot = cx.big + (size_t)cid * need;
  const Group cta{t, NT, 0, sh.redf[0], sh.redi[0]};
  const Team tm{rank * NT + t, C * NT, rank * (NT / 32) + (t >> 5), C * (NT / 32), C, NT / 32, st.redw, st.part,
                st.paddr};
  uint32_t qbase_cl = 0;
  for (int c = 0; c < kClassCluster; ++c) qbase_cl += cx.hdr->n_class[c];
  for (int phase = 0; phase < 2; ++phase) {
    const uint32_t n = phase == 0 ? n_gl : n_cl;
    if (n == 0) continue;
    const int cls = phase == 0 ? kClassGlobal : kClassCluster;
    for (;;) {
      if (rank == 0 && t == 0) st.q = atomicAdd(&cx.hdr->q_next[cls], 1u);
      if (C > 1)
        cl_sync();
      else
        __syncthreads();
      const uint32_t q = C > 1 ? cl_ld_u32(st.qaddr) : st.q;
      if (C > 1)
        cl_sync();  // CTA 0 overwrites q only after every CTA has read it
      else
        __syncthreads();
      if (q >= n) break;
      const int p = (int)cx.queue[(phase == 0 ? 0u : qbase_cl) + q];
      if (phase == 0) {
        run_pair_bwd(cx, bwd_pair(cx, p), reinterpret_cast<float*>(slot), tm, reinterpret_cast<float*>(smem));
      } else {
        const RTeam<true> rt{cta, &st, C, rank};
        run_pair_bwd_r<true>(cx, make_bgeo(cx, p, cc), rt, smem, kBwdSmem, reinterpret_cast<float*>(slot), need,
                             st.rbase);
      }
    }
  }
}

// The resident classes: every CTA on its own drains them by group levels, as
// the forward does (whole CTA, halves, quarters, eighths, warps), each group
// with the slot of its region in the CTA's slot area.  cluster: the cluster
// size the plan classified with.
template <int NT>
__global__ void __launch_bounds__(NT, 1) bwd_res_kernel(CallArgs a, int n_cta, int cluster) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) BwdShared<NT> sh;
  const size_t area = bwd_area_bytes<NT>(a.K);
  bwd_setup(a, sh.cx, sh.om, n_cta, area);
  const BwdCtx& cx = sh.cx;
  const int t = threadIdx.x;
  const ClassCfg cc = bwd_cfg<NT>(cluster);
  if (cx.areas + (size_t)n_cta * area > a.ws + a.ws_bytes) {  // the slot areas must fit
    if (blockIdx.x == 0 && t == 0 && cx.n_pairs > 0) set_status(cx.hdr, 2 /* CF_ERR_WORKSPACE */, -1);
    return;
  }
  const Group cta{t, NT, 0, sh.redf[0], sh.redi[0]};
  unsigned char* area_base = cx.areas + (size_t)blockIdx.x * area;
  const uint64_t ratio = bwd_slot_ratio_q(cx.K, (size_t)cc.z_wrp);
  uint32_t qbase = cx.hdr->n_class[kClassGlobal];
  for (int level = kClassCta; level <= kClassWarp; ++level) {
    Group grp = cta;
    unsigned char* region = smem;
    int slot = 0;
    if (level == kClassHalf) {
      const int hg = t / (NT / 2);
      grp = Group{t % (NT / 2), NT / 2, 5 + hg, sh.redf[1] + hg * (NT / 32), sh.redi[1] + hg * (NT / 32)};
      region = smem + (size_t)hg * cc.z_half;
      slot = 1 + hg;
    } else if (level == kClassQuarter) {
      const int qg = t / (NT / 4);
      grp = Group{t % (NT / 4), NT / 4, 1 + qg, sh.redf[2] + qg * (NT / 64), sh.redi[2] + qg * (NT / 64)};
      region = smem + (size_t)qg * cc.z_qtr;
      slot = 3 + qg;
    } else if (level == kClassEighth) {
      const int eg = t / (NT / 8);
      grp = Group{t % (NT / 8), NT / 8, 7 + eg, sh.redf[3] + eg * (NT / 128), sh.redi[3] + eg * (NT / 128)};
      region = smem + (size_t)eg * cc.z_8th;
      slot = 7 + eg;
    } else if (level == kClassWarp) {
      grp = Group{t & 31, 32, -1, nullptr, nullptr};
      region = smem + (size_t)(t >> 5) * cc.z_wrp;
      slot = 15 + (t >> 5);
    }
    const size_t ro = (size_t)(region - smem);
    float* gslot = reinterpret_cast<float*>(area_base + bwd_slot_at(ro, ratio));
    const size_t gslot_bytes = bwd_slot_at(ro + group_region(level, cc), ratio) - bwd_slot_at(ro, ratio);
    const uint32_t count = cx.hdr->n_class[level];
    for (;;) {
      if (grp.rank == 0) sh.p[slot] = atomicAdd(&cx.hdr->q_next[level], 1u);
      grp.sync();
      const uint32_t q = sh.p[slot];
      grp.sync();
      if (q >= count) break;
      const RTeam<false> rt{grp, nullptr, 1, 0};
      run_pair_bwd_r<false>(cx, make_bgeo(cx, (int)cx.queue[qbase + q], cc), rt, region, group_region(level, cc),
                            gslot, gslot_bytes, nullptr);
    }
    qbase += count;
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

// Per device and variant: the kernels' attributes, the SM count, the resident
// clusters of each size, and the side stream and events of the fork that
// runs the two kernels side by side.
struct BwdDev {
  int n_sm = 0;
  int clusters[kMaxCluster + 1] = {};
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::mutex mu;  // one fork / join sequence at a time (the events are shared)
};

template <int NT>
cudaError_t bwd_init(BwdDev** out) {
  static DeviceOnce once;
  static BwdDev devs[kMaxDevices];
  int dev = 0;
  const cudaError_t e = once.run(
      [](int d) {
        BwdDev& b = devs[d];
        b.n_sm = sm_count_of(d);
        cudaError_t r = cudaFuncSetAttribute(bwd_big_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kBwdSmem);
        if (r == cudaSuccess)
          r = cudaFuncSetAttribute(bwd_res_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
        if (r == cudaSuccess) r = cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking);
        if (r == cudaSuccess) r = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming);
        if (r == cudaSuccess) r = cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming);
        if (r != cudaSuccess) return r;
        if (cudaFuncSetAttribute(bwd_big_kernel<NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
          cudaGetLastError();
        for (int C = 2; C <= kMaxCluster; C *= 2) {
          cudaLaunchConfig_t cfg = {};
          cudaLaunchAttribute attr[1];
          attr[0].id = cudaLaunchAttributeClusterDimension;
          attr[0].val.clusterDim.x = C;
          attr[0].val.clusterDim.y = 1;
          attr[0].val.clusterDim.z = 1;
          cfg.gridDim = dim3(C, 1, 1);
          cfg.blockDim = dim3(NT, 1, 1);
          cfg.dynamicSmemBytes = kBwdSmem;
          cfg.attrs = attr;
          cfg.numAttrs = 1;
          int n = 0;
          if (cudaOccupancyMaxActiveClusters(&n, bwd_big_kernel<NT>, &cfg) != cudaSuccess) n = 0;
          cudaGetLastError();
          b.clusters[C] = n;
        }
        return b.n_sm > 0 ? cudaSuccess : cudaErrorInvalidDevice;
      },
      &dev);
  *out = e == cudaSuccess ? &devs[dev] : nullptr;
  return e;
}

// The large pairs' kernel on the caller's stream, the resident classes'
// kernel on a side stream forked from it and joined back (both capturable in
// a CUDA graph): the large pairs are the critical path and take the SMs first;
// the resident kernel fills the SMs no cluster can use at once and the rest
// as the large pairs finish.
template <int NT>
cudaError_t launch_bwd(const CallArgs& a, int C, cudaStream_t s) {
  BwdDev* d = nullptr;
  cudaError_t e = bwd_init<NT>(&d);
  if (e != cudaSuccess) return e;
  const int n_cl = C >= 2 && C <= kMaxCluster ? d->clusters[C] : 0;
  const int n_res = d->n_sm;  // resident kernel: one CTA per SM, each with a slot area
  bwd_zero_kernel<<<2 * d->n_sm, 256, 0, s>>>(a);
  {
    std::lock_guard<std::mutex> lk(d->mu);
    e = cudaEventRecord(d->fork, s);
    if (e != cudaSuccess) return e;
    if (n_cl > 0) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(n_cl * C, 1, 1);
      cfg.blockDim = dim3(NT, 1, 1);
      cfg.dynamicSmemBytes = kBwdSmem;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, bwd_big_kernel<NT>, a, n_res);
      if (e != cudaSuccess) return e;
    } else {
      bwd_big_kernel<NT><<<d->n_sm, NT, kBwdSmem, s>>>(a, n_res);
    }
    e = cudaStreamWaitEvent(d->side, d->fork, 0);
    if (e != cudaSuccess) return e;
    bwd_res_kernel<NT><<<n_res, NT, kBwdSmem, d->side>>>(a, n_res, n_cl > 0 ? C : 0);
    e = cudaEventRecord(d->join, d->side);
    if (e != cudaSuccess) return e;
    e = cudaStreamWaitEvent(s, d->join, 0);
    if (e != cudaSuccess) return e;
  }
  if (a.grad_w_a) bwd_scatter_kernel<<<2 * d->n_sm, 256, 0, s>>>(a, 0);
  if (a.grad_w_b && a.pack_a != a.pack_b) bwd_scatter_kernel<<<2 * d->n_sm, 256, 0, s>>>(a, 1);
  return cudaGetLastError();
}

template <int NT>
BwdShape bwd_shape_of(int C, int K) {
  BwdShape b{};
  BwdDev* d = nullptr;
  if (bwd_init<NT>(&d) != cudaSuccess) {
    cudaGetLastError();
    return b;
  }
  const int n_cl = C >= 2 && C <= kMaxCluster ? d->clusters[C] : 0;
  b.cluster = n_cl > 0 ? C : 0;
  b.n_cta = d->n_sm;  // the resident kernel's CTAs, one slot area each
  b.n_teams = n_cl > 0 ? n_cl : d->n_sm;
  b.area_bytes = bwd_area_bytes<NT>(K);
  b.cc = bwd_cfg<NT>(b.cluster);
  return b;
}

}  // namespace

BwdShape bwd_shape(int variant, int cluster, int K) {
  return variant == 1 ? bwd_shape_of<512>(cluster, K) : bwd_shape_of<768>(cluster, K);
}

cudaError_t launch_backward(const CallArgs& a, int variant, cudaStream_t s) {
  return variant == 1 ? launch_bwd<512>(a, a.cluster, s) : launch_bwd<768>(a, a.cluster, s);
}

}  // namespace cfsim
