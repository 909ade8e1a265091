// a7: CUDA-graph capture of a sequence of cfsim calls, so that a batch step
// (plan kernels, persistent forward, top-k, ...) replays as one graph launch.
// Host code only.
#include <cuda_runtime.h>

#include <cstdio>
#include <new>

#include "../../include/cfsim.h"

namespace cfsim {
void set_error_detail(const char* msg);
}

struct cf_graph_s {
  cudaGraphExec_t exec;
  int n_nodes;
};

namespace {

cf_status gfail(cf_status s, const char* msg) {
  cfsim::set_error_detail(msg);
  return s;
}

cf_status gcuda(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  cfsim::set_error_detail(buf);
  return CF_ERR_CUDA;
}

}  // namespace

extern "C" {

cf_status cf_graph_begin(cf_stream_t stream) {
  if (!stream) return gfail(CF_ERR_INVALID_ARG, "capture needs a created stream, not the legacy default stream");
  cudaError_t e = cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return gcuda(e, "cf_graph_begin");
  cfsim::set_error_detail("");
  return CF_OK;
}

cf_status cf_graph_end(cf_stream_t stream, cf_graph* out) {
  if (!stream) return gfail(CF_ERR_INVALID_ARG, "stream is NULL");
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
    return gfail(CF_ERR_INVALID_ARG, "the stream is not capturing (no cf_graph_begin)");
  cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &g);  // always ends the capture
  if (!out) {
    if (g) cudaGraphDestroy(g);
    return gfail(CF_ERR_INVALID_ARG, "out is NULL");
  }
  *out = nullptr;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // the failed capture's error must not surface in a later call
    return gcuda(e, "cf_graph_end (a call that cannot be captured ran during the capture)");
  }
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return gcuda(e, "cf_graph_end instantiate");
  cf_graph h = new (std::nothrow) cf_graph_s{x, (int)n};
  if (!h) {
    cudaGraphExecDestroy(x);
    return gfail(CF_ERR_CUDA, "out of host memory");
  }
  *out = h;
  cfsim::set_error_detail("");
  return CF_OK;
}

cf_status cf_graph_launch(cf_graph g, cf_stream_t stream) {
  if (!g) return gfail(CF_ERR_INVALID_ARG, "graph is NULL");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return gcuda(e, "cf_graph_launch");
  cfsim::set_error_detail("");
  return CF_OK;
}

int32_t cf_graph_nodes(cf_graph g) { return g ? g->n_nodes : -1; }

cf_status cf_graph_destroy(cf_graph g) {
  if (!g) return CF_OK;
  cudaError_t e = cudaGraphExecDestroy(g->exec);
  delete g;
  if (e != cudaSuccess) return gcuda(e, "cf_graph_destroy");
  return CF_OK;
}

}  // extern "C"
