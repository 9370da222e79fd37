// Drift-diffusion trials (Sec. 4.4; the DDM nodes of Sec. 5), one thread per
// trial, state in registers:
//   x_j = x_{j-1} + (A dt + sigma sqrt(dt) eps_j), stop at the first j with
//   |x_j| >= z; choice = (x_j > 0), step = j; -1 / max_steps on timeout.
// eps_j is normal j-1 of the (seed, trial, 0) stream, so one Philox block
// feeds four consecutive steps.
//
// Batched form: a persistent grid; when a lane's trial ends it takes the next
// trial id from a global cursor (warp-aggregated atomic), so lanes of a warp
// stay busy although trials end at very different steps.
// Plain form: one thread per trial, one launch, a warp runs until its
// slowest trial ends.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

struct DdmLane {
  float x, c, adt, z;
};

__device__ __forceinline__ void ddm_begin(const DdmParams& p, long long t, DdmLane& s) {
  s.adt = __ldg(p.A + t) * p.dt;
  s.z = __ldg(p.z + t);
  s.x = p.x0;
  s.c = 0.0f;
}

// Up to four steps k .. k+3 of one trial with the four normals of its Philox
// block k / 4. Returns the 1-based sub-step at which the trial crossed a
// bound, or 0.
__device__ __forceinline__ int ddm_four_steps(const DdmParams& p, const float4& e, int k,
                                              DdmLane& s) {
  const float ev[4] = {e.x, e.y, e.z, e.w};
  int hit = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (hit == 0 && k + j < p.max_steps) {
      comp_add(s.x, s.c, fmaf(p.diffusion, ev[j], s.adt));
      if (fabsf(s.x + s.c) >= s.z) hit = j + 1;
    }
  }
  return hit;
}

__device__ __forceinline__ float4 ddm_noise(const DdmParams& p, long long t, int k) {
  return normals4(noise_block(p.k0, p.k1, p.trial0 + (uint32_t)t, 0u, (uint32_t)(k >> 2)));
}

__device__ __forceinline__ void ddm_write(const DdmParams& p, long long t, int hit, int k,
                                          const DdmLane& s) {
  const float xs = s.x + s.c;
  p.choice[t] = hit ? (int8_t)(xs > 0.0f ? 1 : 0) : (int8_t)-1;
  p.step[t] = hit ? k + hit : p.max_steps;
  if (p.xout) p.xout[t] = xs;
}

// Next trial of this lane: f is the value fetched from the cursor.
__device__ __forceinline__ long long ddm_trial(const DdmParams& p, long long f) {
  return p.perm ? (long long)__ldg(p.perm + f) : f;
}

__global__ void __launch_bounds__(256) ddm_batched(DdmParams p) {
  long long f = fetch_trial(p.cursor, true);
  bool active = f >= 0 && f < p.n;
  long long t = active ? ddm_trial(p, f) : 0;
  DdmLane s;
  int k = 0;
  float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) {
    ddm_begin(p, t, s);
    e = ddm_noise(p, t, 0);
  }
  while (__any_sync(kFull, active)) {
    bool finished = false;
    if (active) {
      // the next block's normals do not depend on the state, so they are
      // computed alongside this block's four sequential updates
      const float4 en = ddm_noise(p, t, k + 4);
      const int hit = ddm_four_steps(p, e, k, s);
      if (hit || k + 4 >= p.max_steps) {
        ddm_write(p, t, hit, k, s);
        finished = true;
      } else {
        k += 4;
        e = en;
      }
    }
    f = fetch_trial(p.cursor, finished);
    if (finished) {
      active = f < p.n;
      k = 0;
      if (active) {
        t = ddm_trial(p, f);
        ddm_begin(p, t, s);
        e = ddm_noise(p, t, 0);
      }
    }
  }
}

__global__ void __launch_bounds__(256) ddm_plain(DdmParams p) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  DdmLane s;
  ddm_begin(p, t, s);
  for (int k = 0;; k += 4) {
    const int hit = ddm_four_steps(p, ddm_noise(p, t, k), k, s);
    if (hit || k + 4 >= p.max_steps) {
      ddm_write(p, t, hit, k, s);
      return;
    }
  }
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
    const long long need = (p.n + block - 1) / block;
    if (grid > need) grid = (int)need;
    ddm_batched<<<grid, block, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace dg
