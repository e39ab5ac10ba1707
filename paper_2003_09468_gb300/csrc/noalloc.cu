// Allocation-free walker orthonormalisation (afqmc_orthonormalise_noalloc).
//
// Some callers may not allocate device memory at all: code that runs while a
// CUDA graph is being captured in global mode (where cudaMalloc is an error),
// plug-ins living inside a host application that owns and budgets every device
// byte, or callers that must never fail on memory in the middle of a
// simulation.  For them this file offers a handle-free variant of the
// Householder re-orthonormalisation kernel whose scratch space (the Q factor
// being assembled) is a fixed array in the library's device image instead of a
// cudaMalloc'd buffer.  The array costs every GPU that loads the library
// AFQMC_NOALLOC_SCRATCH_BYTES until the process exits.
#include <mutex>

#include "handle.hpp"

namespace {

constexpr size_t kScratchElems = AFQMC_NOALLOC_SCRATCH_BYTES / sizeof(zc);
constexpr int kMaxDevices = 256;

// File-scope scratch: one copy per device, shared by every call on that device.
static __device__ __align__(256) zc g_qr_scratch[kScratchElems];

std::mutex g_mu;
zc* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in: the kernel must receive the address returned by
// cudaGetSymbolAddress, resolved once per device with that device current.
cudaError_t scratch_address(zc** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qr_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<zc*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" afqmc_status afqmc_orthonormalise_noalloc(void* phi, int rows, int cols, int nmat, void* stream) {
  if (!phi || rows < 1 || cols < 1 || cols > rows || cols > 1024 || nmat < 1) return AFQMC_ERR_INVALID;
  // the kernel moves (re, im) pairs as 16-byte vectors: refuse an 8-byte-aligned C array here
  // instead of letting the device fault on it
  if (reinterpret_cast<uintptr_t>(phi) & 15u) return AFQMC_ERR_INVALID;
  if ((size_t)rows * (size_t)cols * (size_t)nmat > kScratchElems) return AFQMC_ERR_INVALID;
  zc* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return AFQMC_ERR_CUDA;
  // The kernel writes every scratch entry it reads (it starts the Q factor from
  // the identity), so nothing left by an earlier call leaks into this one.
  e = fp64::qr_launch(static_cast<zc*>(phi), scratch, rows, cols, nmat, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? AFQMC_OK : AFQMC_ERR_CUDA;
}
