// Small networks, one lane per trial, with the DDM nodes of the Extended
// Stroop run after the network in the same lane (the kernel templates are in
// dg_net_lane.cuh).
#include "dg_net_lane.cuh"

namespace dg {

cudaError_t launch_net_lane_ext(const NetParams& p, const NetDense& q, cudaStream_t s) {
  return launch_lane<false, true>(p, q, nullptr, s);
}

}  // namespace dg
