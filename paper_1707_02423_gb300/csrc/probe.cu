// On-chip peaks the rooflines are quoted against: shared-memory, L2 and
// distributed-shared-memory load bandwidth and the FP32 FMA rate, each
// measured by a kernel that does nothing else, with the SM clock of the same
// launch read from clock64 / %globaltimer so that the result can be expressed
// per clock per SM and rescaled to the clock another kernel ran at.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "../../include/cfsim.h"
#include "layout.h"

namespace cfsim {
void set_error_detail(const char* msg);
}

namespace {

using cfsim::align_up;

constexpr int kNT = 1024;        // threads per probe CTA, two CTAs per SM
constexpr int kUnroll = 8;       // independent loads (FMA chains) per loop trip
constexpr int kSmemVec = 2048;   // uint4 slots per CTA (32 KB)
constexpr int kL2Words = 4;      // words per thread of the L2 buffer (loads in flight per trip); a power of two

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 of each CTA records the cycles and nanoseconds the CTA's timed
// loop took.
struct BlockClock {
  long long c0;
  unsigned long long t0;
  __device__ __forceinline__ void start() {
    __syncthreads();
    if (threadIdx.x == 0) {
      c0 = clock64();
      t0 = global_ns();
    }
  }
  __device__ __forceinline__ void stop(unsigned long long* clk) {
    __syncthreads();
    if (threadIdx.x == 0) {
      clk[2 * blockIdx.x] = (unsigned long long)(clock64() - c0);
      clk[2 * blockIdx.x + 1] = global_ns() - t0;
    }
  }
};

__device__ __forceinline__ void keep(uint32_t acc, uint32_t* sink) {
  if (acc == 0x9e3779b9u) *sink = acc;  // practically never true; keeps the loads live
}

// Each warp reads 32 consecutive 16-byte words (512 contiguous bytes: four
// conflict-free wavefronts) per load.
__global__ void __launch_bounds__(kNT, 2) probe_smem_kernel(int iters, uint32_t* sink, unsigned long long* clk) {
  __shared__ __align__(16) uint4 buf[kSmemVec];
  for (int k = threadIdx.x; k < kSmemVec; k += kNT) buf[k] = make_uint4(k, 3 * k, 5 * k, 7 * k);
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
  uint32_t acc = 0;
  BlockClock bc;
  bc.start();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t idx = (threadIdx.x + (uint32_t)(it * kUnroll + u) * 32u) & (kSmemVec - 1);
      uint32_t x, y, z, w;
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                   : "r"(base + idx * 16u));
      acc ^= (x ^ y) ^ (z ^ w);
    }
  }
  bc.stop(clk);
  keep(acc, sink);
}

// Every thread re-reads its kL2Words words of an L2-resident buffer (one word
// per grid stride) with volatile loads, which bypass L1.
__global__ void __launch_bounds__(kNT, 2) probe_l2_kernel(const uint4* __restrict__ buf, int passes, uint32_t* sink,
                                                          unsigned long long* clk) {
  const size_t gs = (size_t)gridDim.x * kNT;
  const size_t g = (size_t)blockIdx.x * kNT + threadIdx.x;
  uint32_t acc = 0;
  BlockClock bc;
  bc.start();
  for (int it = 0; it < passes; ++it) {
#pragma unroll
    for (int u = 0; u < kL2Words; ++u) {
      // volatile loads: each one is performed (ordinary loads of an unchanging
      // buffer may be merged across passes), and they are served by L2, not L1
      const size_t idx = g + (size_t)((it + u) & (kL2Words - 1)) * gs;
      uint32_t x, y, z, w;
      asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                   : "l"(buf + idx)
                   : "memory");
      acc ^= (x ^ y) ^ (z ^ w);
    }
  }
  bc.stop(clk);
  keep(acc, sink);
}

__global__ void probe_fill_kernel(uint4* buf, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    buf[k] = make_uint4((uint32_t)k, (uint32_t)(k >> 7), 0x5bd1e995u, (uint32_t)(3 * k));
}

// Two-CTA clusters: every thread reads the partner CTA's shared memory
// through its cluster address (mapa + ld.shared::cluster).  The cluster
// barriers before and after the loop make the partner's buffer valid and keep
// it alive while it is read; both CTAs of a cluster are co-scheduled, so the
// barriers always complete.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kNT, 2)
    probe_dsmem_kernel(int iters, uint32_t* sink, unsigned long long* clk) {
  __shared__ __align__(16) uint4 buf[kSmemVec];
  for (int k = threadIdx.x; k < kSmemVec; k += kNT) buf[k] = make_uint4(k, 3 * k, 5 * k, 7 * k);
  uint32_t rank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const uint32_t local = (uint32_t)__cvta_generic_to_shared(buf);
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank ^ 1u));
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  uint32_t acc = 0;
  BlockClock bc;
  bc.start();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t idx = (threadIdx.x + (uint32_t)(it * kUnroll + u) * 32u) & (kSmemVec - 1);
      uint32_t x, y, z, w;
      asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                   : "r"(remote + idx * 16u));
      acc ^= (x ^ y) ^ (z ^ w);
    }
  }
  bc.stop(clk);
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  keep(acc, sink);
}

// kUnroll independent FMA chains per thread.
__global__ void __launch_bounds__(kNT, 2) probe_fp32_kernel(int iters, float a, float b, uint32_t* sink,
                                                            unsigned long long* clk) {
  float x[kUnroll];
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) x[u] = (float)(threadIdx.x + u);
  BlockClock bc;
  bc.start();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) x[u] = fmaf(x[u], a, b);
  }
  bc.stop(clk);
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) s += x[u];
  keep(__float_as_uint(s), sink);
}

struct ProbeLayout {
  size_t clk, sink, buf, total;
  size_t buf_vec;  // uint4 words of the L2 buffer
  int grid;
};

ProbeLayout probe_layout(int kind, int n_sm) {
  ProbeLayout L{};
  L.grid = 2 * n_sm;
  size_t o = 0;
  L.clk = o;
  o = align_up(o + 16 * (size_t)L.grid, 256);
  L.sink = o;
  o = align_up(o + 4, 256);
  L.buf = o;
  if (kind == CF_PROBE_L2) {
    L.buf_vec = (size_t)L.grid * kNT * kL2Words;  // 128 KB per SM: 19 MB on 152 SMs, well inside L2
    o = align_up(o + 16 * L.buf_vec, 256);
  }
  L.total = o;
  return L;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cf_status err(cf_status s, const char* msg) {
  cfsim::set_error_detail(msg);
  return s;
}

cf_status cuda_err(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  cfsim::set_error_detail(buf);
  return CF_ERR_CUDA;
}

}  // namespace

extern "C" {

cf_status cf_probe_ws_size(int32_t kind, size_t* bytes) {
  if (!bytes) return err(CF_ERR_INVALID_ARG, "bytes is NULL");
  if (kind < CF_PROBE_SMEM || kind > CF_PROBE_FP32) return err(CF_ERR_INVALID_ARG, "unknown probe kind");
  const int n_sm = sm_count();
  if (n_sm <= 0) return err(CF_ERR_CUDA, "no CUDA device");
  *bytes = probe_layout(kind, n_sm).total;
  cfsim::set_error_detail("");
  return CF_OK;
}

cf_status cf_probe(int32_t kind, void* d_ws, size_t ws_bytes, int32_t reps, cf_stream_t stream,
                   cf_probe_result* out) {
  if (!out || !d_ws) return err(CF_ERR_INVALID_ARG, "d_ws and out are required");
  if (kind < CF_PROBE_SMEM || kind > CF_PROBE_FP32) return err(CF_ERR_INVALID_ARG, "unknown probe kind");
  if (reps < 1 || reps > 1000) return err(CF_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  const int n_sm = sm_count();
  if (n_sm <= 0) return err(CF_ERR_CUDA, "no CUDA device");
  const ProbeLayout L = probe_layout(kind, n_sm);
  if (ws_bytes < L.total) return err(CF_ERR_WORKSPACE, "probe workspace too small (see cf_probe_ws_size)");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(d_ws);
  unsigned long long* clk = reinterpret_cast<unsigned long long*>(base + L.clk);
  uint32_t* sink = reinterpret_cast<uint32_t*>(base + L.sink);
  uint4* buf = reinterpret_cast<uint4*>(base + L.buf);
  // iteration counts sized for launches of several milliseconds at about 2 GHz
  const int iters = kind == CF_PROBE_FP32 ? 65536 : kind == CF_PROBE_L2 ? 4096 : 8192;
  double work = 0.0;
  const double threads = (double)L.grid * kNT;
  if (kind == CF_PROBE_SMEM || kind == CF_PROBE_DSMEM) work = threads * iters * kUnroll * 16.0;
  if (kind == CF_PROBE_L2) work = (double)L.buf_vec * 16.0 * iters;
  if (kind == CF_PROBE_FP32) work = threads * iters * kUnroll * 2.0;

  cudaError_t e = cudaSuccess;
  if (kind == CF_PROBE_L2) {
    probe_fill_kernel<<<L.grid, 256, 0, st>>>(buf, L.buf_vec);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "probe fill");
  }
  auto launch = [&]() -> cudaError_t {
    switch (kind) {
      case CF_PROBE_SMEM: probe_smem_kernel<<<L.grid, kNT, 0, st>>>(iters, sink, clk); break;
      case CF_PROBE_L2: probe_l2_kernel<<<L.grid, kNT, 0, st>>>(buf, iters, sink, clk); break;
      case CF_PROBE_DSMEM: probe_dsmem_kernel<<<L.grid, kNT, 0, st>>>(iters, sink, clk); break;
      default: probe_fp32_kernel<<<L.grid, kNT, 0, st>>>(iters, 1.0000001f, 1e-7f, sink, clk); break;
    }
    return cudaGetLastError();
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_err(e, "probe events");
  }
  std::vector<unsigned long long> h(2 * (size_t)L.grid);
  double best = 1e30, best_mhz = 0.0;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // launch 0 warms up
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
    if ((e = launch()) != cudaSuccess) break;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h.data(), clk, 16 * (size_t)L.grid, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (r == 0 || ms >= best) continue;
    std::vector<double> mhz;
    for (int b = 0; b < L.grid; ++b)
      if (h[2 * b + 1] > 0) mhz.push_back(1e3 * (double)h[2 * b] / (double)h[2 * b + 1]);
    std::sort(mhz.begin(), mhz.end());
    best = ms;
    best_mhz = mhz.empty() ? 0.0 : mhz[mhz.size() / 2];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_err(e, "probe launch");
  out->work = work;
  out->best_ms = best;
  out->rate = work / (best * 1e-3);
  out->sm_mhz = best_mhz;
  out->per_clk_sm = best_mhz > 0.0 ? out->rate / (best_mhz * 1e6 * n_sm) : 0.0;
  out->n_sm = n_sm;
  cfsim::set_error_detail("");
  return CF_OK;
}

}  // extern "C"
