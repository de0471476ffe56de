// One-time kernel attributes, per device.  cudaFuncSetAttribute applies to
// the current device only, so a launcher records, per device ordinal, that
// it has raised a kernel's dynamic shared-memory limit there; a launch on a
// device seen for the first time sets the attribute again.
#pragma once

#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

namespace be {

// Raise the dynamic shared-memory limit of `func` to `bytes` on the current
// device unless `done` (the caller's record for this kernel, one bit per
// device ordinal below 64) says it was raised there already.  Concurrent
// first calls may both set the attribute, which is harmless; ordinals of 64
// and above set it on every call.
inline cudaError_t smem_limit_once(const void *func, int bytes, std::atomic<uint64_t> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t)1 << dev : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace be
