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
enum { CF_MATCH_GREEDY = 0,  /* greedy: largest remaining entry first (the default)      */
       CF_MATCH_OPTIMAL = 1  /* maximum-weight assignment of min(n_a, n_b) pairs (the
                                "best matching" alternative; Hungarian method, one warp
                                per pair); needs the matrices (d_X), CFGs <= 9000 blocks */ };

/* flags */
enum {
  CF_FLAG_PER_PAIR_LAUNCH = 1u << 0, /* one kernel launch per pair, no batching: the plain
                                        form the batched path is measured against           */
  CF_FLAG_PLAN_ONLY = 1u << 1,       /* run only the device-side plan of the pair list (cost
                                        order, offsets) into the workspace                  */
  CF_FLAG_REUSE_PLAN = 1u << 2,      /* skip the plan: reuse the one a previous call with the
                                        same packs, pairs and workspace left there          */
  CF_FLAG_OPT_UNSTAGED = 1u << 3,    /* testing: under CF_MATCH_OPTIMAL every matrix is read
                                        from global memory instead of being staged in the
                                        kernel's shared-memory slot pool -- the path a warp
                                        takes when its bounded wait for slots runs out       */
  CF_FLAG_PER_PAIR_STREAMS = 1u << 4 /* with CF_FLAG_PER_PAIR_LAUNCH: the launches are spread
                                        over 32 streams forked from the caller's stream and
                                        joined back to it (pair p on stream p mod 32, each
                                        stream with its own scratch slot), so launches of the
                                        plain form no longer run one after another; for
                                        measuring what the batched form's gain is made of    */
};

typedef struct cf_params {
  float alpha;        /* restart blend, 0 <= alpha < 1 (default 0.8)            */
  int32_t K;          /* iterations, K >= 0 (default 40)                         */
  int32_t norm_mode;  /* CF_NORM_FROB (default) or CF_NORM_NONE                   */
  int32_t match_mode; /* CF_MATCH_GREEDY (default) or CF_MATCH_OPTIMAL               */
  uint32_t flags;     /* CF_FLAG_*                                                */
  int32_t tune;       /* kernel configuration: 0 = built-in default, else an id in
                         [1, cf_num_tunes()] (cf_autotune picks one)              */
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
 * copies.  A larger workspace is fine.  params->tune matters: the tunes whose
 * matching steps are deferred (cf_tune_info.matching 3) need 6 more bytes per
 * X entry, which this adds; size with the tune the call will use. */
cf_status cf_similarity_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                                const cf_params* params, size_t* bytes);

/* ---- a2-a7: similarity, matching, score ---------------------------------- */
/* For every pair: steps above up to X_K; optionally the greedy matching and
 * graph score.  d_pack_a may equal d_pack_b.  d_pairs: int32 [P, 2] on the
 * device.  d_omega: float [F] on the device, >= 0.  Outputs (each may be NULL):
 * d_X (layout above), d_scores [P], d_match (layout above).  All pairs run in
 * one batched, load-balanced pass (persistent kernels pulling pairs from a
 * cost-ordered queue) unless params->flags has CF_FLAG_PER_PAIR_LAUNCH.
 * With params->match_mode == CF_MATCH_OPTIMAL the matching and score are the
 * maximum-weight assignment on the written d_X, which is then required.
 * P == 0 is a no-op. */
cf_status cf_similarity(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                        const cf_params* params, const float* d_omega, float* d_X, float* d_scores,
                        int32_t* d_match, void* d_ws, size_t ws_bytes, cf_stream_t stream);

/* Node matching and graph score.  With d_X_in == NULL the similarity is
 * recomputed (same as cf_similarity with d_match / d_scores).  With d_X_in
 * given (layout of cf_similarity's d_X) only the matching runs on those
 * matrices: greedy, or the maximum-weight assignment when params is given
 * with match_mode CF_MATCH_OPTIMAL (params is otherwise unused and may be
 * NULL, as may d_omega).  A pair with a CFG above 9000 blocks under
 * CF_MATCH_OPTIMAL is skipped and the status word gets CF_ERR_UNSUPPORTED. */
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

/* The winners' pair list of a top-k, on the device, so that their matchings
 * can follow the top-k in the same stream (and the same CUDA graph) without a
 * host round trip: for query q < Q and rank r < k,
 *   d_pairs[2 (q k + r)]     = d_rows ? d_rows[q] : q   (the query's CFG in pack A)
 *   d_pairs[2 (q k + r) + 1] = d_idx[q k + r]           (the winner's CFG in pack B)
 * d_idx: int32 [Q, k] (cf_topk's indices); d_rows: int32 [Q] or NULL; d_pairs:
 * int32 [Q k, 2], caller-owned.  Size the matching call's workspace with
 * cf_similarity_ws_size_any (the pairs are not on the host). */
cf_status cf_topk_pairs(const int32_t* d_idx, int32_t Q, int32_t k, const int32_t* d_rows, int32_t* d_pairs,
                        cf_stream_t stream);

/* Workspace bytes cf_similarity / cf_match need for ANY list of P pairs of
 * these two packs (host copies): an upper bound of cf_similarity_ws_size for
 * pair lists that exist only on the device (e.g. from cf_topk_pairs).  It
 * sizes every pair as the two packs' largest CFGs. */
cf_status cf_similarity_ws_size_any(const void* h_pack_a, const void* h_pack_b, int32_t P, const cf_params* params,
                                    size_t* bytes);

/* ---- the element-wise distances of Table 1 --------------------------------- */
/* The paper's other family of measures (Sec. 4, 4.1, Table 1): the smaller
 * CFG's transition matrix (T[s, d] = weight of edge s -> d, duplicates added)
 * is resized by bilinear interpolation to N = max(n_a, n_b) -- output index t
 * samples the source at t (n - 1) / (N - 1), so corners are kept; a 1 x 1
 * matrix stays constant; equal sizes are not resized -- and five distances
 * are taken between the two N x N matrices x (resized) and y:
 *   CF_DIST_EUCLIDEAN  sqrt(sum (x - y)^2)
 *   CF_DIST_MANHATTAN  sum |x - y|
 *   CF_DIST_MINKOWSKI  (sum |x - y|^p)^(1/p)
 *   CF_DIST_JACCARD    sum (x - y)^2 / (sum x^2 + sum y^2 - sum x y)   (0 if the
 *                      denominator is 0)
 *   CF_DIST_COSINE     1 - sum x y / (|x| |y|)   (0 if both norms are 0, 1 if one is)
 * With CF_DIST_SCALE01 every distance is min-max scaled to [0, 1] over the
 * call's P pairs (Sec. 5.2: 0 = strongest similarity; a constant distance
 * scales to 0).  d_out: float [P][5] in the order above.  0 < p <= 64.  CFGs
 * up to 28,000 blocks (larger: status word CF_ERR_UNSUPPORTED); a pair index
 * out of range: status word CF_ERR_INVALID_ARG (read with cf_status_check on
 * d_ws).  d_ws: cf_distances_ws_size bytes. */
enum { CF_DIST_EUCLIDEAN = 0, CF_DIST_MANHATTAN = 1, CF_DIST_MINKOWSKI = 2, CF_DIST_JACCARD = 3, CF_DIST_COSINE = 4,
       CF_DIST_COUNT = 5 };
enum { CF_DIST_SCALE01 = 1u };
cf_status cf_distances_ws_size(int32_t P, size_t* bytes);
cf_status cf_distances(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P, float p,
                       uint32_t flags, float* d_out, void* d_ws, size_t ws_bytes, cf_stream_t stream);

/* ---- Ward clustering of similarity profiles -------------------------------- */
/* Sec. 5.3 groups kernels with Ward's minimum-variance method on squared
 * Euclidean distances between points.  A CFG's point is its row of the
 * all-pairs score matrix (its similarity profile); cf_score_matrix builds that
 * matrix from a pair list and its scores.
 *
 * cf_score_matrix: zero d_S [n_rows x n_cols] (row-major), then
 * S[a][b] = d_scores[p] for every pair p = (a, b) of d_pairs, and S[b][a] too
 * when symmetric (n_rows == n_cols).  *d_status (one int32 on the device)
 * becomes 0, or 1 + the index of a pair out of range (that pair is skipped).
 *
 * cf_ward: agglomerative Ward clustering of n points d_points [n x dim]
 * (row-major), n <= 16384: n - 1 merges in scipy's linkage convention --
 * merge k joins clusters d_merge[2k] < d_merge[2k+1] (ids below n are points,
 * n + k the cluster formed at merge k) at height d_height[k] (the Ward
 * distance, sqrt of the Lance-Williams-updated squared distance) into
 * d_size[k] points.  Ties: the pair of smallest (slot, slot) index.  Runs the
 * distance matrix on the whole GPU, then the merges on one CTA (L2-resident
 * matrix, per-row minimum cache).  d_ws: cf_ward_ws_size bytes (4 n^2 + O(n));
 * its first word is a status word (cf_status_check): CF_ERR_NUMERIC if the
 * points hold NaN. */
cf_status cf_score_matrix(const int32_t* d_pairs, const float* d_scores, int32_t P, int32_t n_rows, int32_t n_cols,
                          int32_t symmetric, float* d_S, int32_t* d_status, cf_stream_t stream);
cf_status cf_ward_ws_size(int32_t n, size_t* bytes);
cf_status cf_ward(const float* d_points, int32_t n, int32_t dim, int32_t* d_merge, float* d_height, int32_t* d_size,
                  void* d_ws, size_t ws_bytes, cf_stream_t stream);

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
 *   - params->flags may not hold CF_FLAG_PLAN_ONLY or CF_FLAG_REUSE_PLAN
 *     (CF_ERR_INVALID_ARG): every call plans afresh, because a plan kept in
 *     the shared array can be replaced by any other call in between.
 *   - All calls share the array; each call clears what must start at zero.
 *     Calls whose device work can overlap (other streams without ordering)
 *     race on the array and give wrong results.
 *   - The first call on a device resolves the array's address
 *     (cudaGetSymbolAddress, that device current): make it before any stream
 *     capture begins. */
cf_status cf_similarity_noalloc(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs, int32_t P,
                                const cf_params* params, const float* d_omega, float* d_X, float* d_scores,
                                int32_t* d_match, int32_t* d_status, cf_stream_t stream);

/* ---- a7: autotuner --------------------------------------------------------- */
/* Kernel configurations of the batched forward, by tune id (cf_params.tune):
 * threads per CTA (1024, 768 or 512), the smallest thread group a pair may be
 * given (a warp, an eighth, quarter or half CTA, or the whole CTA), the matching
 * policy of shared-memory-resident pairs (ranked lists wherever their state
 * fits, only in groups of at most a quarter CTA, or never: rounds of
 * rescans; or, ids 181-240, ranked lists wherever they fit with the greedy's
 * sequential steps run by a second kernel, one warp per pair, on lists the
 * forward leaves in the workspace: 6 bytes per X entry of every pair, which
 * cf_similarity_ws_size adds for these ids; a workspace without that room
 * makes the forward run the steps itself), and the cluster
 * tier: pairs too large for one CTA split by rows over the 2, 4 or 8 CTAs of
 * a thread-block cluster with the iterates in distributed shared memory (or,
 * with no cluster tier, iterated by one CTA out of L2).  Every tune gives the
 * same results up to rounding; only the speed differs. */
typedef struct cf_tune_info {
  int32_t tune;
  int32_t threads_per_cta; /* 1024, 768 or 512                                */
  int32_t smallest_group;  /* threads: 32, or threads_per_cta / 8, / 4, / 2, / 1 */
  int32_t matching;        /* 0 ranked where it fits, 1 ranked in groups of at
                              most a quarter CTA, 2 rescans only, 3 ranked where
                              it fits with the steps deferred to a second
                              kernel                                            */
  int32_t cluster;         /* CTAs per thread-block cluster of the cluster tier
                              (0: none; pairs too large for one CTA then use the
                              global-memory tier)                               */
} cf_tune_info;
int32_t cf_num_tunes(void);
cf_status cf_tune_describe(int32_t tune, cf_tune_info* out);

/* Workspace bytes cf_autotune needs for this pair list (host copies). */
cf_status cf_autotune_ws_size(const void* h_pack_a, const void* h_pack_b, const int32_t* h_pairs, int32_t P,
                              const cf_params* params, size_t* bytes);

/* Pick the fastest tune for this workload: time cf_similarity (scores and
 * matchings) under every tune on a deterministic sample of at most 16384 of
 * the pairs (pair floor(k P / S), k < S), one warm-up and three timed calls
 * each, and return the fastest in *tune (its time in *best_ms, may be NULL).
 * When one call of the default tune on the sample takes over 40 ms, the
 * candidates are timed on an evenly strided part of it that fits 40 ms; over
 * 160 ms (pairs of hundreds to thousands of blocks), on the whole sample,
 * once each, and only the thread counts and cluster sizes (smallest group a
 * warp, matching policy 1), the other choices not mattering for such pairs.
 * The choice is cached in the text file cache_path (or, when NULL, in the file
 * named by the environment variable CF_AUTOTUNE_CACHE; no caching if neither
 * is set) under a key of device name, SM count, F_pad, K, norm_mode and the
 * sample's cost distribution; a cache hit returns at once without device work.
 * Host copies (h_pack_*, h_pairs) size and key the run, device copies run it.
 * BLOCKS.  d_ws: cf_autotune_ws_size bytes, contents overwritten. */
cf_status cf_autotune(const void* h_pack_a, const void* h_pack_b, const void* d_pack_a, const void* d_pack_b,
                      const int32_t* h_pairs, int32_t P, const cf_params* params, const float* d_omega, void* d_ws,
                      size_t ws_bytes, const char* cache_path, cf_stream_t stream, int32_t* tune, float* best_ms);

/* ---- a7: CUDA-graph capture --------------------------------------------- */
/* A batch step (plan kernels, persistent forward, top-k, matching of the
 * winners, ...) recorded once and replayed as one graph launch, so the
 * per-step cost is one host call whatever the number of kernels.
 *   cf_graph_begin(stream)      starts capturing `stream` (thread-local mode);
 *                               `stream` must be a created stream, not NULL
 *   ... cfsim calls that enqueue on `stream` (cf_similarity, cf_match,
 *       cf_similarity_backward, cf_topk) ...
 *   cf_graph_end(stream, &g)    ends the capture and instantiates it; fails
 *                               with CF_ERR_CUDA if a call that cannot be
 *                               captured ran in between (anything documented
 *                               as BLOCKS, e.g. cf_status_check, cf_pack_cfgs)
 *   cf_graph_launch(g, stream)  replays on any stream (same pointers, same
 *                               sizes: the buffers named while capturing must
 *                               stay allocated while g exists)
 *   cf_graph_destroy(g)
 * Make one uncaptured call of each kind first: the first use of a kernel
 * sets its attributes, which must not happen during a capture.  The graph
 * handle is host memory owned by the library until cf_graph_destroy. */
typedef struct cf_graph_s* cf_graph;
cf_status cf_graph_begin(cf_stream_t stream);
cf_status cf_graph_end(cf_stream_t stream, cf_graph* out);
cf_status cf_graph_launch(cf_graph g, cf_stream_t stream);
/* Nodes of the captured graph (kernels and memsets), -1 for NULL. */
int32_t cf_graph_nodes(cf_graph g);
cf_status cf_graph_destroy(cf_graph g);

/* ---- measurement: on-chip peaks ------------------------------------------- */
/* The similarity iterations are bound by on-chip memory, not HBM, so their
 * roofline needs on-chip peaks.  Each probe is a kernel that does only one
 * thing, launched on two CTAs per SM:
 *   CF_PROBE_SMEM   shared-memory loads, 128-bit, conflict-free     (bytes/s)
 *   CF_PROBE_L2     re-reads of an L2-resident buffer (128 KB per SM) with
 *                   volatile loads (L1 bypassed)                     (bytes/s)
 *   CF_PROBE_DSMEM  loads from the partner CTA's shared memory in 2-CTA
 *                   thread-block clusters                            (bytes/s)
 *   CF_PROBE_FP32   independent FP32 FMA chains, 2 FLOPs per FMA     (FLOP/s)
 * The SM clock of the same launch is read on the device (clock64 cycles over
 * %globaltimer nanoseconds, median over CTAs), so per_clk_sm can be rescaled
 * to the clock another kernel ran at. */
enum { CF_PROBE_SMEM = 0, CF_PROBE_L2 = 1, CF_PROBE_DSMEM = 2, CF_PROBE_FP32 = 3 };

typedef struct cf_probe_result {
  double work;       /* bytes (FLOPs) one probe launch moves (computes)            */
  double best_ms;    /* fastest timed launch (CUDA events on the caller's stream)  */
  double rate;       /* work / best_ms, per second                                  */
  double sm_mhz;     /* SM clock during that launch                                 */
  double per_clk_sm; /* rate / (sm_mhz * n_sm): bytes (FLOPs) per clock per SM      */
  int32_t n_sm;      /* SMs of the current device                                   */
} cf_probe_result;

/* Workspace bytes of a probe on the current device (a few hundred bytes; about
 * 19 MB for CF_PROBE_L2 on 152 SMs). */
cf_status cf_probe_ws_size(int32_t kind, size_t* bytes);

/* Run probe `kind` once to warm up and then `reps` times (1..1000) on `stream`,
 * and report the fastest launch.  BLOCKS (synchronises `stream` after every
 * launch).  d_ws: at least cf_probe_ws_size bytes, contents overwritten. */
cf_status cf_probe(int32_t kind, void* d_ws, size_t ws_bytes, int32_t reps, cf_stream_t stream,
                   cf_probe_result* out);

/* ---- status word ---------------------------------------------------------- */
/* Read the device status word of the last call that used d_ws.  BLOCKS
 * (synchronises `stream`).  Returns CF_OK or the first device-side error. */
cf_status cf_status_check(const void* d_ws, cf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CFSIM_H_ */
