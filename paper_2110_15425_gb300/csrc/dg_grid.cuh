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

// The x and y components of the 2-D vectors below go through the paired
// FP32 instructions of this architecture (each component rounded as the
// scalar instruction), so an evaluation keeps its bits.

// unit(v), with unit(v) = 0 for |v|^2 below the smallest normal number (the
// hardware reciprocal square root, flush-to-zero form: a position difference
// that small is zero for this model)
__device__ __forceinline__ float2 unit2(float2 v) {
  const float n2 = v.x * v.x + v.y * v.y;
  if (n2 >= FLT_MIN) {
    const float r = approx_rsqrt(n2);
    return __fmul2_rn(v, f2(r));
  }
  return f2(0.f);
}

// Perception and Action nodes: X^_e = X_e + sd_e eps_{2e+c} (normals 0..5 of
// stream (trial, cand) starting at Philox block block0), then
// act = unit(unit(Y^ - P^) - weight unit(D^ - P^)).
__device__ __forceinline__ float2 pp_act(const PhiloxKeys& rk, uint32_t trial, uint32_t cand,
                                         uint32_t block0, const float* X, float sd0, float sd1,
                                         float sd2, float weight) {
  const float4 z = normals4(noise_block_rk(rk, trial, cand, block0));
  const uint4 w1 = noise_block_rk(rk, trial, cand, block0 + 1u);
  float z4, z5;
  box_muller(w1.x, w1.y, z4, z5);
  const float2 ph = __ffma2_rn(f2(sd0), f2(z.x, z.y), f2(X[0], X[1]));
  const float2 dh = __ffma2_rn(f2(sd1), f2(z.z, z.w), f2(X[2], X[3]));
  const float2 yh = __ffma2_rn(f2(sd2), f2(z4, z5), f2(X[4], X[5]));
  const float2 nph = f2(-ph.x, -ph.y);
  const float2 uy = unit2(__fadd2_rn(yh, nph));
  const float2 ud = unit2(__fadd2_rn(dh, nph));
  return unit2(__ffma2_rn(f2(-weight), ud, uy));
}

// Objective node: -|P + act - Y| - sum_e a_e^2 (cost given), true P and Y.
__device__ __forceinline__ float pp_outcome_at(const PhiloxKeys& rk, uint32_t trial,
                                               uint32_t cand, uint32_t block0, const float* X,
                                               float sd0, float sd1, float sd2, float weight,
                                               float cost) {
  const float2 a = pp_act(rk, trial, cand, block0, X, sd0, sd1, sd2, weight);
  const float2 n = __fadd2_rn(__fadd2_rn(f2(X[0], X[1]), a), f2(-X[4], -X[5]));
  return -approx_sqrt(n.x * n.x + n.y * n.y) - cost;
}

}  // namespace dg
