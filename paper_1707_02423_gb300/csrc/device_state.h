// Per-device host state of the launchers.  Kernel attributes set with
// cudaFuncSetAttribute (the dynamic shared-memory limit, non-portable cluster
// sizes) and queried values (SM count, resident clusters) belong to one
// device, so a process that uses several devices needs them once per device.
// DeviceOnce runs a set-up function once per device, under std::call_once, so
// concurrent first calls from several host threads are safe.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

namespace cfsim {

constexpr int kMaxDevices = 64;

class DeviceOnce {
 public:
  // Runs init(dev) once for the current device dev and returns its result on
  // this and every later call for that device; *dev_out gets dev.
  template <class F>
  cudaError_t run(F&& init, int* dev_out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(flag_[dev], [&] { err_[dev] = init(dev); });
    if (dev_out) *dev_out = dev;
    return err_[dev];
  }

 private:
  std::once_flag flag_[kMaxDevices];
  cudaError_t err_[kMaxDevices] = {};
};

// SM count of device dev (0 on failure, the CUDA error cleared).
inline int sm_count_of(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace cfsim
