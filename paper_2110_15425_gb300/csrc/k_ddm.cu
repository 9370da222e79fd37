// Drift-diffusion trials (Sec. 4.4; the DDM nodes of Sec. 5):
//   x_j = x_{j-1} + (A dt + sigma sqrt(dt) eps_j), stop at the first j with
//   |x_j| >= z; choice = (x_j > 0), step = j; -1 / max_steps on timeout.
// eps_j is normal j-1 of the (seed, trial, 0) stream: Philox block b feeds
// steps 4b .. 4b+3.
//
// The state is kept in 64-bit fixed point with 40 fractional bits: each FP32
// increment is rounded once to a multiple of 2^-40 (an error below 2^-41 per
// step, far under FP32's own) and then summed exactly. Exact sums do not
// depend on their order, which allows the batched form to give a trial a whole
// warp: lane i draws the four increments of block k/4 + i, an int64 warp scan
// places every one of the 128 steps' states, and a ballot finds the first
// crossing. A trial then advances 128 steps per iteration, no lane waits for
// another lane's trial, and the results are bit-identical to the one-thread-
// per-trial plain form, which sums the same integers one step at a time.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

constexpr float kFixScale = 1099511627776.0f;       // 2^40
constexpr float kFixInv = 9.094947017729282e-13f;   // 2^-40

__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * kFixScale); }

__device__ __forceinline__ float from_fix(long long v) { return __ll2float_rn(v) * kFixInv; }

struct DdmTrial {
  float adt;        // A dt
  long long zf;     // threshold, fixed point
  long long x;      // state, fixed point
};

__device__ __forceinline__ DdmTrial ddm_begin(const DdmParams& p, long long t) {
  DdmTrial d;
  d.adt = __ldg(p.A + t) * p.dt;
  d.zf = to_fix(__ldg(p.z + t));
  d.x = to_fix(p.x0);
  return d;
}

__device__ __forceinline__ float4 ddm_noise(const DdmParams& p, long long t, uint32_t block) {
  return normals4(noise_block(p.k0, p.k1, p.trial0 + (uint32_t)t, 0u, block));
}

__device__ __forceinline__ bool crossed(long long x, long long zf) { return x >= zf || x <= -zf; }

__device__ __forceinline__ long long pick(const long long (&v)[4], int i) {
  long long r = v[0];
  r = i == 1 ? v[1] : r;
  r = i == 2 ? v[2] : r;
  r = i == 3 ? v[3] : r;
  return r;
}

__device__ __forceinline__ void ddm_write(const DdmParams& p, long long t, bool hit, int step,
                                          long long x) {
  p.choice[t] = hit ? (int8_t)(x > 0 ? 1 : 0) : (int8_t)-1;
  p.step[t] = hit ? step : p.max_steps;
  if (p.xout) p.xout[t] = from_fix(x);
}

// One trial per warp, 128 steps per iteration (the batched form).
__device__ void ddm_trial_warp(const DdmParams& p, long long t) {
  const int lane = threadIdx.x & 31;
  const DdmTrial d = ddm_begin(p, t);
  long long x = d.x;
  for (int k = 0; k < p.max_steps; k += 128) {
    const float4 e = ddm_noise(p, t, (uint32_t)(k >> 2) + (uint32_t)lane);
    const float ev[4] = {e.x, e.y, e.z, e.w};
    long long pre[4];   // this lane's partial sums after each of its four steps
    long long acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc += to_fix(fmaf(p.diffusion, ev[j], d.adt));
      pre[j] = acc;
    }
    // exclusive scan of the lanes' block sums (exact, so any order is fine)
    long long incl = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    const long long base = x + (incl - acc);
    const int s0 = k + 4 * lane;   // 0-based index of this lane's first step
    int first = 4;
#pragma unroll
    for (int j = 3; j >= 0; --j)
      if (s0 + j < p.max_steps && crossed(base + pre[j], d.zf)) first = j;
    const unsigned hit_lanes = __ballot_sync(kFull, first < 4);
    if (hit_lanes) {
      const int src = __ffs(hit_lanes) - 1;
      if (lane == src) ddm_write(p, t, true, s0 + first + 1, base + pick(pre, first));
      return;
    }
    const int last = p.max_steps - 1 - k;   // step index of max_steps within this chunk
    if (last < 128) {
      // timeout: the state after step max_steps
      const int src = last >> 2;
      if (lane == src) ddm_write(p, t, false, p.max_steps, base + pick(pre, last & 3));
      return;
    }
    x += __shfl_sync(kFull, incl, 31);
  }
}

// Persistent grid: each warp takes the next trial (in the hand-out order)
// until none is left.
__global__ void __launch_bounds__(256) ddm_batched(DdmParams p) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long f = 0;
    if (lane == 0) f = atomicAdd(p.cursor, 1ull);
    f = __shfl_sync(kFull, f, 0);
    if (f >= (unsigned long long)p.n) return;
    const long long t = p.perm ? (long long)__ldg(p.perm + f) : (long long)f;
    ddm_trial_warp(p, t);
  }
}

// One thread per trial, one step at a time (the plain form).
__global__ void __launch_bounds__(256) ddm_plain(DdmParams p) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  const DdmTrial d = ddm_begin(p, t);
  long long x = d.x;
  for (int k = 0; k < p.max_steps; k += 4) {
    const float4 e = ddm_noise(p, t, (uint32_t)(k >> 2));
    const float ev[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (k + j >= p.max_steps) break;
      x += to_fix(fmaf(p.diffusion, ev[j], d.adt));
      if (crossed(x, d.zf)) {
        ddm_write(p, t, true, k + j + 1, x);
        return;
      }
    }
  }
  ddm_write(p, t, false, p.max_steps, x);
}

}  // namespace

int ddm_max_blocks_per_sm(int block) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ddm_batched, block, 0);
  return nb;
}

cudaError_t launch_ddm(const DdmParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  if (mode == 1) {
    const int block = 256;
    const long long grid = (p.n + block - 1) / block;
    ddm_plain<<<(unsigned)grid, block, 0, s>>>(p);
  } else {
    const int block = cfg.block;
    int grid = cfg.grid;
    if (grid <= 0) grid = num_sms() * ddm_max_blocks_per_sm(block);
    const long long need = (p.n * 32 + block - 1) / block;   // one warp per trial
    if (grid > need) grid = (int)need;
    ddm_batched<<<grid, block, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace dg
