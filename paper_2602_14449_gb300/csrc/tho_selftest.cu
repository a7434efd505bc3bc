// Device side of tho_plan_expire_wait: the failure path of the tcgen05
// kernels, exercised without a fault.  Those kernels hand shared-memory stages
// between warps through mbarriers and never wait without a bound: mbar_wait
// gives up after a fixed number of polls, the kernel leaves its loop and
// latches THO_ERR_TIMEOUT in the plan's status word, which the host reads with
// tho_plan_status.  Here one thread waits on a freshly initialized mbarrier
// that nothing arrives at, through the same mbar_wait, with a short bound.
#include <cuda_runtime.h>

#include "tho_launch.h"
#include "tho_umma.cuh"

namespace tho {
namespace {

__global__ void k_expire_wait(int* status, int spins) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  mbar_init(b, 1);  // one expected arrival, which never comes
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(b, 0, spins)) atomicExch(status, 6);  // THO_ERR_TIMEOUT
}

}  // namespace

cudaError_t launch_expire_wait(int* status, int spins, cudaStream_t st) {
  k_expire_wait<<<1, 32, 0, st>>>(status, spins);
  return cudaGetLastError();
}

}  // namespace tho
