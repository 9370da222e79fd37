// Device helpers shared by the predator-prey kernels (grid search, episodes):
// running top-2 argmax summaries and one evaluation of the model (Sec. 2.1).
#pragma once

#include <cfloat>
#include <climits>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

struct GridResultDev {           // dg_grid_result
  long long best_index;
  double best_value;
  double gap;
};

__device__ __forceinline__ TopTwo top_init() { return TopTwo{-DBL_MAX, LLONG_MAX, -DBL_MAX}; }

// Order of doubles as 64-bit integers: for every non-NaN x, y,
// okey(x) < okey(y) exactly when x < y (zero of either sign maps to 0, so the
// two zeros compare equal as they do in IEEE arithmetic). The merges below
// compare and select through these keys on the integer units: the
// double-precision unit of this GPU is a small fraction of its FP32 rate, and
// in the small, latency-bound searches its compares dominated.
__device__ __forceinline__ long long okey(double v) {
  long long b = __double_as_longlong(v);
  if (b == (long long)0x8000000000000000ull) b = 0;
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// Merge two running top-2 summaries: best value with lowest index on ties,
// and the largest value among the rest.
__device__ __forceinline__ TopTwo top_merge(TopTwo a, TopTwo b) {
  const long long ka = okey(a.v1), kb = okey(b.v1);
  const bool b_wins = (kb > ka) || (kb == ka && b.i1 < a.i1);
  TopTwo r;
  if (b_wins) {
    r.v1 = b.v1;
    r.i1 = b.i1;
    r.v2 = okey(a.v1) > okey(b.v2) ? a.v1 : b.v2;
  } else {
    r.v1 = a.v1;
    r.i1 = a.i1;
    r.v2 = okey(b.v1) > okey(a.v2) ? b.v1 : a.v2;
  }
  return r;
}

__device__ __forceinline__ TopTwo top_shfl(TopTwo t, int src, unsigned mask = kFull) {
  TopTwo r;
  r.v1 = __shfl_sync(mask, t.v1, src);
  r.i1 = __shfl_sync(mask, t.i1, src);
  r.v2 = __shfl_sync(mask, t.v2, src);
  return r;
}

__device__ __forceinline__ TopTwo top_warp(TopTwo t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t = top_merge(t, top_shfl(t, (threadIdx.x & 31) ^ o));
  return t;
}

// Candidate sums. Each lane adds its trials' FP32 outcomes into a compensated
// pair (hi, lo): Knuth's TwoSum keeps the rounding error of every addition
// exactly and lo collects them, so hi + lo carries the sum to about 2^-48 of
// its magnitude. The warp combines the pairs the same way and hi + lo is
// converted to FP64 once per candidate, for up to 32 candidates in one
// instruction: the double-precision unit, slow on this GPU, does a handful of
// operations per 32 candidates instead of two per trial.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

// Pair sum over the LANES lanes of a candidate's group, by an xor
// butterfly; every lane of the group ends with the total, added in a fixed
// order.
template <int LANES>
__device__ __forceinline__ void group_pair_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(kFull, hi, o);
    const float ol = __shfl_xor_sync(kFull, lo, o);
    two_sum_add(hi, lo, oh);
    lo += ol;
  }
}

// FP64 mean of a candidate from its pair and 1 / (number of trials).
__device__ __forceinline__ double pair_mean(float hi, float lo, double inv) {
  return ((double)hi + (double)lo) * inv;
}

// Warp total of the lanes' pairs, returned to every lane (tree toward lane 0,
// then broadcast, so every lane holds the same pair).
__device__ __forceinline__ void warp_pair_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_down_sync(kFull, hi, o);
    const float ol = __shfl_down_sync(kFull, lo, o);
    two_sum_add(hi, lo, oh);
    lo += ol;
  }
  hi = __shfl_sync(kFull, hi, 0);
  lo = __shfl_sync(kFull, lo, 0);
}

// unit(v), with unit(v) = 0 for |v|^2 below the smallest normal number (the
// hardware reciprocal square root, flush-to-zero form: a position difference
// that small is zero for this model)
__device__ __forceinline__ void unit2(float vx, float vy, float& ox, float& oy) {
  const float n2 = vx * vx + vy * vy;
  if (n2 >= FLT_MIN) {
    const float r = approx_rsqrt(n2);
    ox = vx * r;
    oy = vy * r;
  } else {
    ox = 0.f;
    oy = 0.f;
  }
}

// Perception and Action nodes: X^_e = X_e + sd_e eps_{2e+c} (normals 0..5 of
// stream (trial, cand) starting at Philox block block0), then
// act = unit(unit(Y^ - P^) - weight unit(D^ - P^)).
__device__ __forceinline__ void pp_act(const PhiloxKeys& rk, uint32_t trial, uint32_t cand,
                                       uint32_t block0, const float* X, float sd0, float sd1,
                                       float sd2, float weight, float& ax, float& ay) {
  const float4 z = normals4(noise_block_rk(rk, trial, cand, block0));
  const uint4 w1 = noise_block_rk(rk, trial, cand, block0 + 1u);
  float z4, z5;
  box_muller(w1.x, w1.y, z4, z5);
  const float phx = fmaf(sd0, z.x, X[0]), phy = fmaf(sd0, z.y, X[1]);
  const float dhx = fmaf(sd1, z.z, X[2]), dhy = fmaf(sd1, z.w, X[3]);
  const float yhx = fmaf(sd2, z4, X[4]), yhy = fmaf(sd2, z5, X[5]);
  float uyx, uyy, udx, udy;
  unit2(yhx - phx, yhy - phy, uyx, uyy);
  unit2(dhx - phx, dhy - phy, udx, udy);
  unit2(fmaf(-weight, udx, uyx), fmaf(-weight, udy, uyy), ax, ay);
}

// Objective node: -|P + act - Y| - sum_e a_e^2 (cost given), true P and Y.
__device__ __forceinline__ float pp_outcome_at(const PhiloxKeys& rk, uint32_t trial,
                                               uint32_t cand, uint32_t block0, const float* X,
                                               float sd0, float sd1, float sd2, float weight,
                                               float cost) {
  float ax, ay;
  pp_act(rk, trial, cand, block0, X, sd0, sd1, sd2, weight, ax, ay);
  const float nx = (X[0] + ax) - X[4];
  const float ny = (X[1] + ay) - X[5];
  return -approx_sqrt(nx * nx + ny * ny) - cost;
}

}  // namespace dg
