// Self-test of the bounded device-side waits (afqmc_kp_wait_selftest).
//
// Every mbarrier wait of the tensor-core kernels goes through tc::mbar_wait,
// which gives up after a cycle limit instead of spinning forever, and the kernel
// that gave up records an error code in the handle's sticky flags.  This entry
// point runs that same wait in a one-warp kernel on an mbarrier that nothing
// else touches, so that a test can make the wait run out on purpose and check
// that the status reaches the host while the context stays usable.  The kernel
// issues no TMA copy and no MMA and holds no tensor memory, so giving up leaves
// nothing in flight.
#include "handle.hpp"
#include "tc.cuh"

namespace {

// One warp.  Lane 0 initialises the barrier for one arrival; with `arrive` set it
// makes that arrival itself (the phase completes and the wait returns at once),
// otherwise nothing arrives and the wait gives up after `limit` cycles.
__global__ void wait_selftest_kernel(int arrive, long long limit, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  __syncwarp();
  if (threadIdx.x == 0) {
    if (arrive) tc::mbar_arrive(&bar);
    if (!tc::mbar_wait(&bar, 0, &abort_flag, limit)) atomicCAS(err, 0, tc::ERR_TIMEOUT_FULL);
  }
  __syncwarp();
}

}  // namespace

extern "C" afqmc_status afqmc_kp_wait_selftest(afqmc_kp_t h, int arrive, long long limit_cycles, void* stream) {
  if (!h || (arrive != 0 && arrive != 1) || limit_cycles < 1 || limit_cycles > (1LL << 31))
    return AFQMC_ERR_INVALID;
  h->launches = 0;
  int* err = h->flags + 1;
  void* args[] = {&arrive, &limit_cycles, &err};
  // cudaLaunchKernel reports this launch's own failure and leaves earlier errors alone
  const cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(wait_selftest_kernel), dim3(1), dim3(32),
                                         args, 0, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return AFQMC_ERR_CUDA;
  AFQMC_LAUNCHED(h);
  return AFQMC_OK;
}
