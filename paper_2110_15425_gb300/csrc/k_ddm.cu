// Drift-diffusion trials (Sec. 4.4; the DDM nodes of Sec. 5):
//   x_j = x_{j-1} + (A dt + sigma sqrt(dt) eps_j), stop at the first j with
//   |x_j| >= z; choice = (x_j > 0), step = j; -1 / max_steps on timeout.
// eps_j is normal j-1 of the (seed, trial, 0) stream: Philox block b feeds
// steps 4b .. 4b+3.
//
// Arithmetic (the same operations in both forms below, so they agree bit for
// bit): inside block b the increments are summed in FP32 in step order,
// p_0 = inc_0, p_j = p_{j-1} + inc_j; the block sums p_3 are rounded once to
// fixed point and added exactly, so the state before block b, X_b, does not
// depend on the order of those additions; the bound test at step j of block b
// is |float(X_b) + p_j| >= z in FP32. A trial whose bound is at most 6 keeps
// X in 32 bits with 28 fractional bits (the states it uses stay below 8 in
// magnitude; sums past a crossing may wrap and are never used); others in 64
// bits with 40. Error against exact arithmetic stays near 1e-6 after 10,000
// steps.
//
// Batched form: one trial per warp, 256 steps per iteration - lane i draws
// blocks k/4 + 2i and k/4 + 2i + 1, an exact warp scan gives every lane its
// X_b, and a ballot finds the first crossing - so no lane waits on another
// lane's trial.
// Plain form: one thread per trial, one block after another.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

// Fixed-point formats of the state: 32 bits with 28 fractional bits (two's
// complement, additions wrap), or 64 bits with 40.
struct Fix32 {
  using T = unsigned int;
  __device__ __forceinline__ static T of(float v) {
    return (T)__float2int_rn(v * 268435456.0f);   // 2^28
  }
  __device__ __forceinline__ static float val(T x) {
    return __int2float_rn((int)x) * 3.7252902984619140625e-9f;   // 2^-28
  }
};
struct Fix64 {
  using T = long long;
  __device__ __forceinline__ static T of(float v) { return to_fix(v); }
  __device__ __forceinline__ static float val(T x) { return from_fix(x); }
};
constexpr float kFix32MaxBound = 6.0f;

struct DdmTrial {
  float adt;        // A dt
  float z;          // threshold
  bool narrow;      // the state fits the 32-bit format
};

__device__ __forceinline__ DdmTrial ddm_begin(const DdmParams& p, long long t) {
  DdmTrial d;
  d.adt = __ldg(p.A + t) * p.dt;
  d.z = __ldg(p.z + t);
  d.narrow = d.z <= kFix32MaxBound && fabsf(p.x0) <= kFix32MaxBound;
  return d;
}

// In-block partial sums p_0 .. p_3 of block `block`.
__device__ __forceinline__ void block_partials(const DdmParams& p, long long t, uint32_t block,
                                               float adt, float (&pre)[4]) {
  const float4 e = normals4(philox_rk(make_uint4(p.trial0 + (uint32_t)t, 0u, block, 0u), p.rk));
  // the four increments A dt + sigma sqrt(dt) eps by two paired fmas (each
  // component rounded as fmaf), then their running sums in order
  const float2 ia = __ffma2_rn(f2(p.diffusion), f2(e.x, e.y), f2(adt));
  const float2 ib = __ffma2_rn(f2(p.diffusion), f2(e.z, e.w), f2(adt));
  pre[0] = ia.x;
  pre[1] = pre[0] + ia.y;
  pre[2] = pre[1] + ib.x;
  pre[3] = pre[2] + ib.y;
}

__device__ __forceinline__ float pick(const float (&v)[4], int i) {
  float r = v[0];
  r = i == 1 ? v[1] : r;
  r = i == 2 ? v[2] : r;
  r = i == 3 ? v[3] : r;
  return r;
}

__device__ __forceinline__ void ddm_write(const DdmParams& p, long long t, bool hit, int step,
                                          float x) {
  p.choice[t] = hit ? (int8_t)(x > 0.0f ? 1 : 0) : (int8_t)-1;
  p.step[t] = hit ? step : p.max_steps;
  if (p.xout) p.xout[t] = x;
}

// One trial per warp, 256 steps per iteration (the batched form): lane i takes
// blocks k/4 + 2i and k/4 + 2i + 1, so the exact scan, the bound ballot and the
// loop run once per 256 steps.
template <typename F>
__device__ __forceinline__ void ddm_trial_warp(const DdmParams& p, long long t,
                                               const DdmTrial& d) {
  using T = typename F::T;
  const int lane = threadIdx.x & 31;
  T x = F::of(p.x0);
  for (int k = 0; k < p.max_steps; k += 256) {
    float pa[4], pb[4];
    const uint32_t b0 = (uint32_t)(k >> 2) + 2u * (uint32_t)lane;
    block_partials(p, t, b0, d.adt, pa);
    block_partials(p, t, b0 + 1u, d.adt, pb);
    const T qa = F::of(pa[3]), q = qa + F::of(pb[3]);
    T incl = q;   // exact scan of the lanes' two-block sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    const T xa_fix = x + (incl - q);
    const float xa = F::val(xa_fix);        // state before this lane's first block
    const float xb = F::val(xa_fix + qa);   // and before its second
    const int s0 = k + 8 * lane;
    // does any of this lane's eight steps reach the bound? (the step cap only
    // matters in the last chunk, a warp-uniform case)
    bool hit;
    if (k + 256 <= p.max_steps) {
      const float m = fmaxf(fmaxf(fmaxf(fabsf(xa + pa[0]), fabsf(xa + pa[1])),
                                  fmaxf(fabsf(xa + pa[2]), fabsf(xa + pa[3]))),
                            fmaxf(fmaxf(fabsf(xb + pb[0]), fabsf(xb + pb[1])),
                                  fmaxf(fabsf(xb + pb[2]), fabsf(xb + pb[3]))));
      hit = m >= d.z;
    } else {
      hit = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hit |= s0 + j < p.max_steps && fabsf(xa + pa[j]) >= d.z;
        hit |= s0 + 4 + j < p.max_steps && fabsf(xb + pb[j]) >= d.z;
      }
    }
    const unsigned hit_lanes = __ballot_sync(kFull, hit);
    if (hit_lanes) {
      if (lane == __ffs(hit_lanes) - 1) {
        int first = 7;
#pragma unroll
        for (int j = 3; j >= 0; --j)
          if (fabsf(xb + pb[j]) >= d.z) first = 4 + j;
#pragma unroll
        for (int j = 3; j >= 0; --j)
          if (fabsf(xa + pa[j]) >= d.z) first = j;
        const float v = first < 4 ? xa + pick(pa, first) : xb + pick(pb, first - 4);
        ddm_write(p, t, true, s0 + first + 1, v);
      }
      return;
    }
    const int last = p.max_steps - 1 - k;   // step index of max_steps within this chunk
    if (last < 256) {
      if (lane == (last >> 3)) {
        const int j = last & 7;
        ddm_write(p, t, false, p.max_steps, j < 4 ? xa + pick(pa, j) : xb + pick(pb, j - 4));
      }
      return;
    }
    x += __shfl_sync(kFull, incl, 31);
  }
}

// Persistent grid: each warp takes the next trial (in the hand-out order)
// until none is left. (40 registers, 6 blocks per SM: the two blocks a lane
// holds spill at the 32 registers of 8 blocks per SM, measured 3 % slower.)
__global__ void __launch_bounds__(256, 6) ddm_batched(DdmParams p) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long f = 0;
    if (lane == 0) f = atomicAdd(p.cursor, 1ull);
    f = __shfl_sync(kFull, f, 0);
    if (f >= (unsigned long long)p.n) return;
    const long long t = p.perm ? (long long)__ldg(p.perm + f) : (long long)f;
    const DdmTrial d = ddm_begin(p, t);
    if (d.narrow)
      ddm_trial_warp<Fix32>(p, t, d);
    else
      ddm_trial_warp<Fix64>(p, t, d);
  }
}

// Several jobs of one model in one launch (the serving loop's groups): each
// warp takes the next entry of the concatenated trial list and runs it as
// ddm_batched does, with its job's inputs, outputs and seed.
__global__ void __launch_bounds__(256, 4) ddm_multi(DdmParams p,
                                                    const __grid_constant__ MultiJobTable tab) {
  __shared__ MultiJob s_job[kMaxMultiJobs];
  copy_jobs(tab, s_job);
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long f = 0;
    if (lane == 0) f = atomicAdd(p.cursor, 1ull);
    f = __shfl_sync(kFull, f, 0);
    if (f >= (unsigned long long)p.n) return;
    const MultiJob& J = s_job[multi_job_of(s_job, tab.n_jobs, (long long)f)];
    DdmParams q = p;
    q.n = J.n;
    q.A = J.in;
    q.z = J.in + J.n;
    q.choice = J.choice;
    q.step = J.step;
    q.xout = J.xout;
    q.trial0 = J.trial0;
    q.rk = philox_keys(J.k0, J.k1);
    const long long t = (long long)f - J.start;
    const DdmTrial d = ddm_begin(q, t);
    if (d.narrow)
      ddm_trial_warp<Fix32>(q, t, d);
    else
      ddm_trial_warp<Fix64>(q, t, d);
  }
}

// One thread per trial, one block after another (the plain form).
template <typename F>
__device__ __forceinline__ void ddm_trial_plain(const DdmParams& p, long long t,
                                                const DdmTrial& d) {
  typename F::T x = F::of(p.x0);
  for (int k = 0; k < p.max_steps; k += 4) {
    float pre[4];
    block_partials(p, t, (uint32_t)(k >> 2), d.adt, pre);
    const float xb = F::val(x);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (k + j >= p.max_steps) break;
      if (fabsf(xb + pre[j]) >= d.z) {
        ddm_write(p, t, true, k + j + 1, xb + pre[j]);
        return;
      }
      if (k + j + 1 == p.max_steps) {
        ddm_write(p, t, false, p.max_steps, xb + pre[j]);
        return;
      }
    }
    x += F::of(pre[3]);
  }
}

__global__ void __launch_bounds__(256) ddm_plain(DdmParams p) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  const DdmTrial d = ddm_begin(p, t);
  if (d.narrow)
    ddm_trial_plain<Fix32>(p, t, d);
  else
    ddm_trial_plain<Fix64>(p, t, d);
}

}  // namespace

int ddm_max_blocks_per_sm(int block) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ddm_batched, block, 0);
  return nb;
}

cudaError_t launch_ddm_multi(const DdmParams& p, const MultiJobTable& tab, cudaStream_t s) {
  if (p.n <= 0 || tab.n_jobs < 1 || tab.n_jobs > kMaxMultiJobs) return cudaErrorInvalidValue;
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ddm_multi, 256, 0);
  if (e != cudaSuccess) return e;
  long long grid = (long long)num_sms() * (nb > 0 ? nb : 1);
  const long long need = (p.n * 32 + 255) / 256;   // one warp per trial
  if (grid > need) grid = need;
  ddm_multi<<<(unsigned)grid, 256, 0, s>>>(p, tab);
  return cudaGetLastError();
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
