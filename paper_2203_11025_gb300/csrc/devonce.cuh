// One-time set-up per device, thread-safe.
//
// A kernel attribute set with cudaFuncSetAttribute (the dynamic shared-memory opt-in,
// non-portable cluster sizes) applies to the device that is current when it is set, so
// caching "done" once per process leaves every other device unconfigured.  DeviceOnce
// keeps the set-up's result per device; the first caller on a device runs it (with that
// device current) under a mutex, later callers read the stored result.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

namespace helm {

struct DeviceOnce {
  static constexpr int kMaxDevices = 64;
  std::mutex mu;
  bool done[kMaxDevices] = {};
  long long value[kMaxDevices] = {};
};

// Runs fn() once per device (the current one) and returns its stored result; returns
// `fail` without calling fn when the current device cannot be read or is out of range.
template <typename F>
long long device_once(DeviceOnce& o, F fn, long long fail = -1) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= DeviceOnce::kMaxDevices) return fail;
  std::lock_guard<std::mutex> lk(o.mu);
  if (!o.done[dev]) {
    o.value[dev] = fn();
    o.done[dev] = true;
  }
  return o.value[dev];
}

// Largest dynamic shared memory a block of `kern` may use on the current device (the
// per-block opt-in limit less the kernel's static shared memory), after raising the
// kernel's limit to it; 0 when any of those calls fails.  Once per device.
template <typename K>
long long opt_in_dynamic_smem(DeviceOnce& o, K kern) {
  return device_once(o, [&]() -> long long {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return optin - (long long)fa.sharedSizeBytes;
  }, 0);
}

// Raises `kern`'s dynamic shared-memory limit to `bytes` once per device; true on success.
template <typename K>
bool set_dynamic_smem(DeviceOnce& o, K kern, int bytes) {
  return device_once(o, [&]() -> long long {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return 1;
  }, 0) == 1;
}

}  // namespace helm
