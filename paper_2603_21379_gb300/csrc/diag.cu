// diag.cu - a kernel that exercises the library's bounded-wait failure path.
//
// Every kernel that waits on an mbarrier (the TMA pipelines of the core and root
// passes) gives up after a poll limit, records a timeout in the handle's device
// status word and returns, so that a lost arrival becomes an RT_ETIMEOUT from
// rt_sync instead of a hung GPU.  k_wait_selftest waits on a barrier that nothing
// arrives on, through the same bounded wait, so the path can be tested without
// faulting or hanging anything.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_common.cuh"
#include "rt_host.h"
#include "tma_util.cuh"

namespace rt {
namespace {

__global__ void k_wait_selftest(int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    tma::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) tma::mbar_wait(&bar, 0, &abort_flag, status);   // phase 0 never completes
  __syncthreads();
}

}  // namespace

cudaError_t diag_set_wait_limit(uint32_t polls) { return tma::set_wait_limit(polls); }

int launch_wait_selftest(int* status, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status);
  return 1;
}

}  // namespace rt
