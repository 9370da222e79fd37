// Self-tests of device building blocks.
//  - The failure path: one CTA waits on an mbarrier that nothing ever arrives
//    on, with the same bounded wait the tensor-core kernel uses, gives up
//    after `limit` cycles and records the expiry in the stream's status word
//    (read back by dg_stream_status). Nothing faults, traps or hangs.
//  - The per-candidate reduction of the grid search and the episodes on given
//    FP32 values: the same lane-group layout, compensated pair sums and FP64
//    mean the kernels apply to their trial outcomes, so that the reduction can
//    be compared on its own with exact sums.
#include "dg_grid.cuh"
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

// Group g of `per` values x[g per .. g per + per - 1] is reduced by LANES
// lanes exactly as a candidate's trial outcomes are: lane l of the group adds
// values l, l + LANES, ... into its pair, the group combines the pairs, and
// the mean is formed in FP64.
template <int LANES>
__global__ void __launch_bounds__(256) pair_sum_kernel(const float* x, long long n_groups,
                                                       int per, double* means) {
  const int lane = threadIdx.x & 31, gl = lane % LANES;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long g = warp * (32 / LANES) + lane / LANES;
  float hi = 0.f, lo = 0.f;
  if (g < n_groups)
    for (int j = gl; j < per; j += LANES) two_sum_add(hi, lo, x[g * per + j]);
  group_pair_sum<LANES>(hi, lo);
  if (g < n_groups && gl == 0) means[g] = pair_mean(hi, lo, 1.0 / (double)per);
}

}  // namespace

cudaError_t launch_pair_sum(const float* x, long long n_groups, int per, int lanes,
                            double* means, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  const long long groups_per_block = 8LL * (32 / lanes);
  const long long grid = (n_groups + groups_per_block - 1) / groups_per_block;
  if (grid > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  if (lanes == 8)
    pair_sum_kernel<8><<<(unsigned)grid, 256, 0, s>>>(x, n_groups, per, means);
  else if (lanes == 32)
    pair_sum_kernel<32><<<(unsigned)grid, 256, 0, s>>>(x, n_groups, per, means);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_wait_timeout(long long limit_cycles, int* status, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(limit_cycles, status);
  return cudaGetLastError();
}

}  // namespace dg
