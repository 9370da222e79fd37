// Small networks, one lane per trial, several jobs in one launch through a job
// table (the kernel templates are in dg_net_lane.cuh).
#include "dg_net_lane.cuh"

namespace dg {

cudaError_t launch_net_lane_multi(const NetParams& p, const NetDense& q, const MultiJobTable& tab,
                                  cudaStream_t s) {
  if (p.n <= 0 || tab.n_jobs < 1 || tab.n_jobs > kMaxMultiJobs) return cudaErrorInvalidValue;
  if (p.n_ddm != 0 || q.n_ddm != 0 || p.cursor == nullptr) return cudaErrorInvalidValue;
  return launch_lane<true, false>(p, q, &tab, s);
}

}  // namespace dg
