// Dynamic shared-memory opt-in, set once per (kernel, device).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

// Raises cudaFuncAttributeMaxDynamicSharedMemorySize of `fn` on the current device to
// `bytes` if it is not already at least that, so that steady-state calls (and calls made
// while a stream is being captured into a graph) issue no attribute call at all.
inline cudaError_t ensure_dyn_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& d = done[{fn, dev}];
  if (bytes <= d) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) d = bytes;
  return e;
}
