// Per-device dynamic shared-memory limits of the kernels that need more than 48 KB.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

namespace sox {

// Raises a kernel's dynamic shared-memory limit once per device: the attribute belongs to
// the device that is current when it is set, so a process driving several GPUs needs it
// on each.  `mask` is the call site's record of the devices done (ordinals below 64).
template <class Kernel>
inline cudaError_t set_smem_once(Kernel *k, int bytes, std::atomic<unsigned long long> &mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (mask.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) mask.fetch_or(bit);
  return e;
}

}  // namespace sox
