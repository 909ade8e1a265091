// Host-side launchers of the kernels (implemented in the .cu files), called by
// the C-ABI layer.  All launches are asynchronous on the given stream and make
// no allocation.
#pragma once

#include <cuda_runtime.h>

#include "layout.h"

namespace cfsim {

// Arguments of one similarity / matching / backward call.
struct CallArgs {
  const void* pack_a;
  const void* pack_b;
  const int32_t* pairs;
  int P;
  float alpha;
  int K;
  int norm_mode;
  const float* omega;
  float* X;        // optional output
  float* scores;   // optional output
  int32_t* match;  // optional output
  const float* X_in;  // cf_match on given matrices
  unsigned char* ws;
  size_t ws_bytes;
  // backward
  const int32_t* match_in;
  const float* grad_scores;
  float* grad_w_a;
  float* grad_w_b;
  float* grad_omega;
  // kernel configuration (the tune of cf_params)
  int min_cls;  // smallest group level of the batched forward
  int ranked;   // matching policy of resident pairs (ClassCfg::ranked)
  int cluster;  // CTAs per cluster of the cluster tier, 0 = none
  int opt_unstaged;  // optimal matching: skip the shared-memory slot pool (CF_FLAG_OPT_UNSTAGED)
  int pp_streams;    // the plain per-pair form: streams its launches are spread over (0/1: the caller's)
};

// Streams the plain per-pair form may be spread over (CF_FLAG_PER_PAIR_STREAMS).
constexpr int kPerPairStreams = 32;

// Batched forward kernel variants: 0 = 1024 threads per CTA, 1 = 512, 2 = 768.
int num_fwd_variants();
// Class configuration of variant v with the given smallest group level,
// matching policy and cluster size.
ClassCfg fwd_class_cfg(int v, int min_cls, int ranked, int cluster);
// C if clusters of C CTAs of variant v can be resident on this device, else 0.
int cluster_supported(int v, int C);

// Kernel configuration selected by cf_params.tune (see decode_tune): ids
// 1..180 enumerate variant x smallest group x matching policies 0-2 x cluster
// size, ids 181..240 the same with matching policy 3 (deferred steps).
constexpr int kNumTunes = 240;
constexpr int kFirstDeferTune = 181;
struct Tune {
  int variant, min_cls, ranked, cluster;
};
Tune decode_tune(int32_t id);

// a7: device-side plan: validate pairs, classify, cost-order them into the
// queue, and compute the X / match offsets.
cudaError_t launch_plan(const CallArgs& a, const ClassCfg& cc, cudaStream_t s);

// a2-a6: the batched persistent forward (or one launch per pair).
cudaError_t launch_forward(const CallArgs& a, int variant, bool per_pair, cudaStream_t s);

// The deferred sequential steps of the greedy matching (matching policy 3):
// one warp per pair whose ranked lists the forward left in the workspace.
cudaError_t launch_match_deferred(const CallArgs& a, cudaStream_t s);

// Greedy matching + score on caller-given matrices.
cudaError_t launch_match_only(const CallArgs& a, cudaStream_t s);

// Maximum-weight assignment + score on the matrices a.X_in (the plan must have
// run); CFGs of up to opt_max_blocks() blocks.
cudaError_t launch_match_optimal(const CallArgs& a, cudaStream_t s);
int opt_max_blocks();

// Pack weight update from user-order weights (pointers into a device pack).
cudaError_t launch_set_weights(CfAdj* out_adj, CfAdj* in_adj, const int32_t* in_eid, const int32_t* u2c,
                               int64_t n_user_edges, int64_t n_edges, const float* w_user, cudaStream_t s);

// a8: adjoint (workspace layout bwd_layout, then the per-CTA slot areas of
// the resident tier, then the per-team slots of the cluster and global tiers;
// the plan must have run with the adjoint's class configuration bwd_shape().cc).
// variant: 1 = 512 threads per CTA, else 768; a.cluster: CTAs per cluster of
// the cluster tier (0 none), as bwd_shape() reported it.
struct BwdShape {
  int cluster;        // CTAs per cluster actually launched (0: none)
  int n_cta;          // CTAs of the launch (one slot area each)
  int n_teams;        // teams that run cluster- or global-class pairs (one slot each at most)
  size_t area_bytes;  // slot area per CTA
  ClassCfg cc;        // classification of the pairs
};
BwdShape bwd_shape(int variant, int cluster, int K);
cudaError_t launch_backward(const CallArgs& a, int variant, cudaStream_t s);

// The element-wise Table 1 distances of resized transition matrices
// (workspace dist_ws_bytes(); CFGs up to dist_max_blocks() blocks).
constexpr int kNumDist = 5;
size_t dist_ws_bytes();
int dist_max_blocks();
cudaError_t launch_distances(const void* pack_a, const void* pack_b, const int32_t* pairs, int P, float p, bool scale,
                             float* out, void* ws, cudaStream_t s);

// Top-k per row.
cudaError_t launch_topk(const float* scores, int Q, int C, int k, float* top, int32_t* idx, cudaStream_t s);
// The winners' pair list from top-k indices.
cudaError_t launch_topk_pairs(const int32_t* idx, int Q, int k, const int32_t* rows, int32_t* pairs, cudaStream_t s);


}  // namespace cfsim
