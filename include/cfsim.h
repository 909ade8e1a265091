/*
 * cfsim -- pairwise control-flow-graph similarity for GPU-kernel subgraph
 * matching, on one GB300 (sm_103a).  C ABI of libcfsim.so.
 *
 * The measure (paper arXiv:1707.02423, "A Similarity Measure for GPU Kernel
 * Subgraph Matching"):
 *   - Table 1, "Cos" row (Sec. 4.2): attribute term, in similarity form,
 *       E_ij = sum_f w_f a_if b_jf / (r_i c_j),  r_i = sqrt(sum_f w_f a_if^2),
 *       c_j = sqrt(sum_f w_f b_jf^2),  E_ij = 0 when r_i c_j = 0,
 *     on per-block attributes (Sec. 1, 3.1: instruction-operation mix,
 *     registers allocated, block execution frequency) with per-feature
 *     weights w = omega.
 *   - Ehat = E / |E|_F (uniform 1/sqrt(n_a n_b) when |E|_F = 0), X_0 = Ehat.
 *   - Table 1, "Iso" row, (I - alpha Q x P) x, read as the IsoRank iteration
 *     (cited in Sec. 2 and 4.2) with Q, P the two CFGs' weighted adjacency
 *     operators (edge weight = transition probability, Sec. 3.1):
 *       Z_k     = 1/2 (W_A X_k W_B^T + W_A^T X_k W_B)
 *       Y_{k+1} = alpha Z_k + (1 - alpha) Ehat
 *       X_{k+1} = Y_{k+1} / |Y_{k+1}|_F,          k = 0 .. K-1 (no early stop)
 *   - Node matching: greedy on X_K (largest entry first; ties by smaller
 *     block index of A, then of B), min(n_a, n_b) pairs.
 *   - Graph score s = sum of X_K over the matched entries (Sec. 5.2 reports
 *     IsoRank scores of 1.00 to 1.30: an unnormalised sum, higher = closer).
 *
 * Conventions for every call below.
 *   - Ownership: the caller owns all memory.  The library never allocates
 *     device memory; it uses only the workspace the caller sizes with the
 *     *_ws_size queries.  Host arrays are borrowed for the duration of a call.
 *   - Streams: device work is enqueued on the caller's stream and returns
 *     without synchronising, except where a call says it blocks.  The
 *     enqueueing calls make no allocation and no synchronisation, so they can
 *     be captured into a CUDA graph once the library has been used once on
 *     the device (first use caches device properties and kernel attributes).
 *   - Errors: every call returns a cf_status; nothing aborts and no C++
 *     exception crosses the ABI.  cf_last_error_detail() gives a message for
 *     the calling thread's last failure.  Faults found on the device (bad
 *     omega, a pair index out of range, a workspace too small for a pair)
 *     are recorded in a status word inside the workspace and read back with
 *     cf_status_check().
 *   - Layout of per-pair outputs (pair p = (pairs[2p], pairs[2p+1]), CFG
 *     pairs[2p] of pack A against CFG pairs[2p+1] of pack B, n_a x n_b):
 *       X:     row-major n_a x n_b matrix at float offset
 *              x_off[p] = sum_{q<p} n_a(q) n_b(q)
 *       match: n_a int32 entries at offset m_off[p] = sum_{q<p} n_a(q);
 *              match[m_off[p] + i] = matched block of B, or -1
 *       score: one float per pair.
 *     cf_out_sizes() gives the totals.
 */
#ifndef CFSIM_H_
#define CFSIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t.  NULL means the legacy default stream. */
typedef struct CUstream_st* cf_stream_t;

typedef enum cf_status {
  CF_OK = 0,
  CF_ERR_INVALID_ARG = 1,  /* bad pointer, size, index, or non-finite / negative value */
  CF_ERR_WORKSPACE = 2,    /* workspace or output buffer smaller than required        */
  CF_ERR_UNSUPPORTED = 3,  /* valid input this build cannot run (e.g. a CFG > 32000 blocks) */
  CF_ERR_CUDA = 4,         /* a CUDA runtime call failed (no device, launch failure)   */
  CF_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out                      */
  CF_ERR_NUMERIC = 6       /* a non-finite value appeared on the device (e.g. in omega) */
} cf_status;

enum { CF_NORM_FROB = 0, /* X_{k+1} = Y_{k+1} / |Y_{k+1}|_F (the method)                */
       CF_NORM_NONE = 1  /* X_{k+1} = Y_{k+1}: plain fixed-point iteration of the Table 1
                            linear system (I - alpha M) x = (1 - alpha) vec Ehat; for tests */ };
enum { CF_MATCH_GREEDY = 0 };

/* flags */
enum {
  CF_FLAG_PER_PAIR_LAUNCH = 1u << 0, /* one kernel launch per pair, no batching: the plain
                                        form the batched path is measured against           */
  CF_FLAG_PLAN_ONLY = 1u << 1,       /* run only the device-side plan of the pair list (cost
                                        order, offsets) into the workspace                  */
  CF_FLAG_REUSE_PLAN = 1u << 2       /* skip the plan: reuse the one a previous call with the
                                        same packs, pairs and workspace left there          */
};

typedef struct cf_params {
  float alpha;        /* restart blend, 0 <= alpha < 1 (default 0.8)            */
  int32_t K;          /* iterations, K >= 0 (default 40)                         */
  int32_t norm_mode;  /* CF_NORM_FROB (default) or CF_NORM_NONE                   */
  int32_t match_mode; /* CF_MATCH_GREEDY                                          */
  uint32_t flags;     /* CF_FLAG_*                                                */
} cf_params;

/* One CFG on the host: blocks 0..n_blocks-1, edges src[e] -> dst[e] with weight
 * w[e] >= 0 (a transition probability, Sec. 3.1), attributes attr[n_blocks x F]
 * row-major, all >= 0 and finite.  Duplicate edges are allowed and add up;
 * self-loops are allowed. */
typedef struct cf_cfg_view {
  int32_t n_blocks;   /* >= 1, <= 32000 */
  int32_t n_edges;    /* >= 0 */
  const int32_t* src; /* [n_edges] */
  const int32_t* dst; /* [n_edges] */
  const float* w;     /* [n_edges] */
  const float* attr;  /* [n_blocks * F] */
} cf_cfg_view;

/* Summary of a pack, read from its header (host copy). */
typedef struct cf_pack_info {
  int32_t n_cfgs;
  int32_t F;            /* attributes per block                        */
  int32_t F_pad;        /* row stride of the attribute matrix (F rounded up to 4) */
  int32_t max_blocks;   /* largest CFG                                  */
  int64_t n_blocks;     /* blocks over all CFGs                         */
  int64_t n_edges;      /* distinct edges over all CFGs (duplicates merged) */
  int64_t n_user_edges; /* edges as given (sum of n_edges of the views) */
  int64_t bytes;        /* total pack size                              */
} cf_pack_info;

/* ---- status ------------------------------------------------------------- */
const char* cf_status_string(cf_status s);
/* Message for the calling thread's last failing call ("" if none).  The
 * pointer stays valid until that thread's next cfsim call. */
const char* cf_last_error_detail(void);
int32_t cf_abi_version(void);

/* ---- a1: CSR batch pack -------------------------------------------------- */
/* Bytes a pack of these CFGs takes (same on host and device).  Validates the
 * views (indices in range, finite nonnegative weights and attributes). */
cf_status cf_pack_size(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, size_t* bytes);

/* Build the pack into host memory h_pack[bytes].  The pack is position
 * independent (offsets, no pointers): the same bytes are valid on the device.
 * Layout: header; per-CFG block / distinct-edge / user-edge offsets; out-CSR
 * (row pointers, {local neighbour, weight} sorted by (src, dst)); in-CSR
 * (sorted by (dst, src)) with the distinct-edge id of each entry; the
 * distinct-edge id of every user edge; attributes [n_blocks x F_pad] float,
 * zero-padded.  Every section starts on a 256-byte boundary. */
cf_status cf_pack_host(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, void* h_pack, size_t bytes);

/* Read a pack header (host copy of a pack). */
cf_status cf_pack_info_get(const void* h_pack, cf_pack_info* info);

/* Build the pack on the host and copy it to d_pack[bytes] on `stream`.
 * BLOCKS until the copy has completed (the host staging buffer is freed). */
cf_status cf_pack_cfgs(const cf_cfg_view* cfgs, int32_t n_cfgs, int32_t F, void* d_pack, size_t bytes,
                       cf_stream_t stream);

/* Overwrite the edge weights of a device pack from user-order weights
 * d_w_user[n_user_edges] (duplicates add up), on `stream`.  Lets the weights be
 * trainable tensors while the graph structure stays fixed. */
cf_status cf_pack_set_weights(void* d_pack, const void* h_pack, const float* d_w_user, cf_stream_t stream);

/* ---- sizes -------------------------------------------------------------- */
/* Total X floats and match int32 entries for a pair list (host arrays). */
cf_status cf_out_sizes(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                       int64_t* x_elems, int64_t* match_elems);

/* Workspace bytes cf_similarity / cf_match need for this pair list.  Uses host
 * copies of the packs and pairs only to size; the device calls take device
 * copies.  A larger workspace is fine. */
cf_status cf_similarity_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                                const cf_params* params, size_t* bytes);

/* ---- a2-a7: similarity, matching, score ---------------------------------- */
/* For every pair: steps above up to X_K; optionally the greedy matching and
 * graph score.  d_pack_a may equal d_pack_b.  d_pairs: int32 [P, 2] on the
 * device.  d_omega: float [F] on the device, >= 0.  Outputs (each may be NULL):
 * d_X (layout above), d_scores [P], d_match (layout above).  All pairs run in
 * one batched, load-balanced pass (persistent kernels pulling pairs from a
 * cost-ordered queue) unless params->flags has CF_FLAG_PER_PAIR_LAUNCH.
 * P == 0 is a no-op. */
cf_status cf_similarity(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                        const cf_params* params, const float* d_omega, float* d_X, float* d_scores,
                        int32_t* d_match, void* d_ws, size_t ws_bytes, cf_stream_t stream);

/* Greedy matching and graph score.  With d_X_in == NULL the similarity is
 * recomputed (same as cf_similarity with d_match / d_scores).  With d_X_in
 * given (layout of cf_similarity's d_X) only the matching runs on those
 * matrices; params and d_omega are then unused and may be NULL. */
cf_status cf_match(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                   const cf_params* params, const float* d_omega, const float* d_X_in, int32_t* d_match,
                   float* d_scores, void* d_ws, size_t ws_bytes, cf_stream_t stream);

/* ---- a8: adjoint --------------------------------------------------------- */
/* Workspace bytes for cf_similarity_backward (includes the per-pair
 * checkpoint store: X every ceil(sqrt(K)) steps). */
cf_status cf_similarity_backward_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs,
                                         int32_t P, const cf_params* params, size_t* bytes);

/* Gradients of sum_p g[p] * s_p with the matching d_match held fixed (the
 * matching of a forward call), with respect to every user edge weight of pack A
 * (d_grad_w_a, [n_user_edges(A)]) and pack B, and to omega (d_grad_omega, [F]).
 * Accumulates (+=) into the caller's buffers.  When d_pack_a == d_pack_b,
 * d_grad_w_b may be NULL (everything goes to d_grad_w_a) or equal d_grad_w_a.
 * Recomputes the forward from checkpoints (every ceil(sqrt(K)) steps). */
cf_status cf_similarity_backward(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                                 const cf_params* params, const float* d_omega, const int32_t* d_match,
                                 const float* d_grad_scores, float* d_grad_w_a, float* d_grad_w_b,
                                 float* d_grad_omega, void* d_ws, size_t ws_bytes, cf_stream_t stream);

/* ---- a9: top-k ----------------------------------------------------------- */
/* For each of Q rows of d_scores [Q, C] (row-major): the k largest scores in
 * descending order (ties: smaller column first) -> d_top [Q, k], d_idx [Q, k].
 * 1 <= k <= C, k <= 1024. */
cf_status cf_topk(const float* d_scores, int32_t Q, int32_t C, int32_t k, float* d_top, int32_t* d_idx,
                  cf_stream_t stream);

/* ---- no-allocation variant ------------------------------------------------- */
/* cf_similarity without a workspace argument, for callers that cannot
 * allocate device memory (code running under an allocator that owns the whole
 * device heap, inside host callbacks, or in a serving loop that must not add
 * allocation latency).  The paper has no counterpart; this is a library
 * convenience.  The workspace is a file-scope 32 MiB device array that every
 * GPU loading the library holds until exit; nothing is allocated per call.
 * Same arguments and outputs as cf_similarity, plus d_status: when not NULL,
 * one int32 on the device that receives this call's device status word
 * (a cf_status code) in stream order.
 *   - A pair list whose fixed workspace part (about 20 bytes per pair) does
 *     not fit in 32 MiB is rejected with CF_ERR_WORKSPACE before any launch;
 *     pairs too large for shared memory need scratch slots from the rest of
 *     the array, and *d_status is CF_ERR_WORKSPACE if none fits.
 *   - All calls share the array; each call clears what must start at zero.
 *     Calls whose device work can overlap (other streams without ordering)
 *     race on the array and give wrong results.
 *   - The first call on a device resolves the array's address
 *     (cudaGetSymbolAddress, that device current): make it before any stream
 *     capture begins. */
cf_status cf_similarity_noalloc(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                                const cf_params* params, const float* d_omega, float* d_X, float* d_scores,
                                int32_t* d_match, int32_t* d_status, cf_stream_t stream);

/* ---- status word ---------------------------------------------------------- */
/* Read the device status word of the last call that used d_ws.  BLOCKS
 * (synchronises `stream`).  Returns CF_OK or the first device-side error. */
cf_status cf_status_check(const void* d_ws, cf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CFSIM_H_ */
