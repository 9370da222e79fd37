// Self-test of the device-side failure path: one CTA waits on an mbarrier that
// nothing ever arrives on, with the same bounded wait the tensor-core kernel
// uses, gives up after `limit` cycles and records the expiry in the stream's
// status word (read back by dg_stream_status). Nothing faults, traps or hangs.
#include "dg_internal.h"
#include "dg_tc.cuh"

namespace dg {

namespace {

__global__ void wait_timeout_kernel(long long limit, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0, limit) && threadIdx.x == 0) atomicExch(status, 1);
}

}  // namespace

cudaError_t launch_wait_timeout(long long limit_cycles, int* status, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(limit_cycles, status);
  return cudaGetLastError();
}

}  // namespace dg
