// Device helpers shared by the small-network kernels (k_net.cu: the lane-group
// and plain forms; k_net_lane.cu: the one-lane form): the clamped inputs' part
// of a unit's net input, and the state of a DDM node (Extended Stroop).
#pragma once

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

__device__ __forceinline__ float const_net(const NetParams& p, int n_in, long long t, int u) {
  const long long g = (long long)p.trial0 + t;  // global trial id
  const int cond = (int)((g / p.cond_block) % p.n_cond);
  const float* cin = p.cond + (size_t)cond * n_in;
  const float* w = p.w_in + (size_t)u * n_in;
  float acc = 0.f;
  for (int q = 0; q < n_in; ++q) acc = fmaf(__ldg(w + q), __ldg(cin + q), acc);
  return acc;
}

struct DdmNode {
  float adt, diff, z;
  int max;
  long long X;      // state before block b, fixed point
  int b;
};

}  // namespace dg
