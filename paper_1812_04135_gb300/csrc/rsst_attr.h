// Raising a kernel's dynamic shared-memory limit is a per-device setting:
// it is applied once on each device that launches the kernel (the caller
// keeps one mask per kernel; bit d = done on device d).
#pragma once

#include <atomic>
#include <cuda_runtime.h>

namespace rsst {

template <class K>
inline cudaError_t set_smem_limit_once(K kern, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

}  // namespace rsst
