// Small networks, one lane per trial: one job, no DDM nodes (the kernel
// templates are in dg_net_lane.cuh).
#include "dg_net_lane.cuh"

namespace dg {

cudaError_t launch_net_lane_ext(const NetParams& p, const NetDense& q, cudaStream_t s);

cudaError_t launch_net_lane(const NetParams& p, const NetDense& q, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  if (p.n_ddm != q.n_ddm || p.cursor == nullptr) return cudaErrorInvalidValue;
  if (q.n_ddm > 0) return launch_net_lane_ext(p, q, s);
  return launch_lane<false, false>(p, q, nullptr, s);
}

}  // namespace dg
