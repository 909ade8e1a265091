// cf_similarity_noalloc: cf_similarity for callers that cannot allocate
// device memory.  Some callers run where cudaMalloc is off limits: inside a
// host callback or a pre-allocated arena, under a custom allocator that owns
// the whole device heap, or in code that must not add allocation latency or
// fragmentation to a serving loop.  This entry point takes no workspace: it
// uses one file-scope device array that every GPU loading this library holds
// until the process exits.
//
// Limits and sharing:
//   - kStaticWsBytes (32 MiB) per device.  The fixed part of the workspace
//     grows with the pair count (about 20 bytes per pair); a call whose pair
//     list alone needs more is rejected on the host with CF_ERR_WORKSPACE.
//     Pairs too large for shared memory take scratch slots from the rest of
//     the array; if not even one slot fits, the device status word reports
//     CF_ERR_WORKSPACE (copied to *d_status when given).
//   - Every call uses the same array and leaves its contents behind.  The
//     call clears the part that must start at zero (the workspace header) on
//     its stream.  Calls whose device work overlaps (different streams, no
//     ordering between them) race on the array and give wrong results.
//   - CF_FLAG_PLAN_ONLY and CF_FLAG_REUSE_PLAN are rejected with
//     CF_ERR_INVALID_ARG: a plan left in the shared array by one call is not
//     safe for a later one.
//   - The first call on a device resolves the array's device address with
//     cudaGetSymbolAddress (that device current).  Make that first call before
//     any stream capture begins.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cfsim.h"
#include "kernels.h"
#include "layout.h"

namespace cfsim {
void set_error_detail(const char* msg);  // api.cu
}

namespace {

constexpr size_t kStaticWsBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// The workspace of cf_similarity_noalloc.  In host code this name is only a
// stand-in for the symbol: never pass it to a kernel; pass the address
// cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_static_ws on the current device (resolved once per device).
cf_status static_ws_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    cfsim::set_error_detail("cf_similarity_noalloc: no usable current CUDA device");
    return CF_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      cfsim::set_error_detail("cf_similarity_noalloc: cudaGetSymbolAddress of the static workspace failed");
      return CF_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CF_OK;
}

}  // namespace

extern "C" cf_status cf_similarity_noalloc(const void* d_pack_a, const void* d_pack_b, const int32_t* d_pairs,
                                           int32_t P, const cf_params* params, const float* d_omega, float* d_X,
                                           float* d_scores, int32_t* d_match, int32_t* d_status,
                                           cf_stream_t stream) {
  // The plan flags would let a call run on a plan an earlier call left in the
  // shared array; any other call in between (another pair list, another user
  // of the library) replaces that plan, and offsets sized for other pairs
  // could then write outside this caller's outputs.  Every call plans afresh.
  if (params && (params->flags & (CF_FLAG_PLAN_ONLY | CF_FLAG_REUSE_PLAN))) {
    cfsim::set_error_detail(
        "cf_similarity_noalloc: CF_FLAG_PLAN_ONLY and CF_FLAG_REUSE_PLAN are not accepted (the static workspace "
        "is shared by every call, so a kept plan cannot be relied on)");
    return CF_ERR_INVALID_ARG;
  }
  if (P > 0 && cfsim::ws_layout(P).fixed_bytes > kStaticWsBytes) {
    cfsim::set_error_detail(
        "cf_similarity_noalloc: the pair list needs more workspace than the 32 MiB static array holds; "
        "split it or use cf_similarity with a caller-sized workspace");
    return CF_ERR_WORKSPACE;
  }
  void* ws = nullptr;
  cf_status s = static_ws_address(&ws);
  if (s != CF_OK) return s;
  s = cf_similarity(d_pack_a, d_pack_b, d_pairs, P, params, d_omega, d_X, d_scores, d_match, ws, kStaticWsBytes,
                    stream);
  if (s == CF_OK && d_status) {
    // the first word of the workspace is the device status of this call (an
    // empty pair list leaves the workspace untouched and reports CF_OK)
    cudaError_t e = P > 0 ? cudaMemcpyAsync(d_status, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                            (cudaStream_t)stream)
                          : cudaMemsetAsync(d_status, 0, sizeof(int32_t), (cudaStream_t)stream);
    if (e != cudaSuccess) {
      cfsim::set_error_detail("cf_similarity_noalloc: status copy failed");
      return CF_ERR_CUDA;
    }
  }
  return s;
}
