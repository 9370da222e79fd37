// Longest-expected-first trial order for the persistent kernels.
//
// A persistent launch ends when its last trial ends. Trials of a DDM or LCA
// job differ in length by more than an order of magnitude, and a long trial
// fetched late keeps a few lanes busy long after the rest of the GPU has run
// dry. Handing trials out in decreasing order of their expected length
// (the classic longest-processing-time-first rule) puts the long ones at the
// front and leaves short trials for the drain. The order only changes which
// lane runs a trial, never its result: every draw is keyed by the trial id.
//
// Expected length keys (in steps, clamped to max_steps):
//   DDM: mean decision time (z / A) tanh(A z / sigma^2) / dt  (Sec. 4.2 asks for
//        exactly this kind of convergence-time estimate);
//   LCA: noise-free time for an accumulator with input I_eff to reach the
//        threshold alone, -ln(1 - k thr / I_eff) / (k dt) (never, max_steps, when
//        I_eff <= k thr), with I_eff = I_max - w mean_{j != max} I_j and
//        w = beta (N - 1) / (1 + beta (N - 1)): the leader's input less the
//        competition. Its rank correlation with the trials' actual lengths is
//        0.85 / 0.72 / 0.58 for N = 4 / 8 / 16 on the inputs U[0, 1] (0.75 / 0.47 /
//        0.25 for I_max alone).
// Keys fall into kBuckets buckets; a three-kernel counting sort (histogram,
// scan, scatter) writes the permutation. Order inside a bucket is arbitrary.
// Each trial's bucket is computed once (by the histogram kernel) and stored,
// so the scatter places exactly the trials the histogram counted.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

constexpr int kSortBlock = 256;
constexpr int kPerThread = 16;

__device__ __forceinline__ int bucket_of(float expected_steps, int max_steps) {
  // bucket 0 = longest
  float f = expected_steps / (float)max_steps;
  f = fminf(fmaxf(f, 0.f), 1.f);
  int b = (int)((1.0f - f) * (float)(kSchedBuckets - 1) + 0.5f);
  return b < 0 ? 0 : (b >= kSchedBuckets ? kSchedBuckets - 1 : b);
}

__device__ __forceinline__ int key_bucket(const SchedParams& s, long long t) {
  float e;
  if (s.kind == 0) {  // DDM
    const float A = fabsf(__ldg(s.a + t)), z = __ldg(s.b + t);
    if (A < 1e-12f) {
      e = (float)s.max_steps;
    } else if (s.sigma2 <= 0.f) {
      e = z / A / s.dt;
    } else {
      e = (z / A) * tanhf(A * z / s.sigma2) / s.dt;
    }
  } else {  // LCA
    const float* I = s.a + (size_t)t * s.N;
    float im = __ldg(I), sum = im;
    for (int i = 1; i < s.N; ++i) {
      const float v = __ldg(I + i);
      im = fmaxf(im, v);
      sum += v;
    }
    if (s.N > 1) {
      // the leader's input less the others' mean input weighted by
      // beta (N - 1) / (1 + beta (N - 1)): the competition it has to overcome
      const float bn = s.inhibition * (float)(s.N - 1);
      im -= bn / (1.0f + bn) * ((sum - im) / (float)(s.N - 1));
    }
    const float kt = s.leak * s.threshold;
    if (im <= kt || im <= 0.f) {
      e = (float)s.max_steps;
    } else if (s.leak > 0.f) {
      e = -log1pf(-kt / im) / (s.leak * s.dt);
    } else {
      e = s.threshold / (im * s.dt);
    }
  }
  return bucket_of(e, s.max_steps);
}

__global__ void __launch_bounds__(kSortBlock) sched_hist(SchedParams s) {
  __shared__ unsigned int h[kSchedBuckets];
  for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortBlock * kPerThread;
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const long long t = base + (long long)j * kSortBlock + threadIdx.x;
    if (t < s.n) {
      const int b = key_bucket(s, t);
      s.bucket[t] = (unsigned short)b;
      atomicAdd(&h[b], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&s.hist[i], h[i]);
}

// exclusive scan of the histogram into the bucket cursors (one block)
__global__ void __launch_bounds__(kSchedBuckets) sched_scan(SchedParams s) {
  __shared__ unsigned int v[kSchedBuckets];
  const int i = threadIdx.x;
  v[i] = s.hist[i];
  __syncthreads();
  for (int off = 1; off < kSchedBuckets; off <<= 1) {
    const unsigned int add = i >= off ? v[i - off] : 0u;
    __syncthreads();
    v[i] += add;
    __syncthreads();
  }
  s.cursor[i] = v[i] - s.hist[i];
}

__global__ void __launch_bounds__(kSortBlock) sched_scatter(SchedParams s) {
  __shared__ unsigned int h[kSchedBuckets];
  __shared__ unsigned int start[kSchedBuckets];
  for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortBlock * kPerThread;
  int bk[kPerThread];
  unsigned int rank[kPerThread];
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const long long t = base + (long long)j * kSortBlock + threadIdx.x;
    bk[j] = -1;
    if (t < s.n) {
      bk[j] = s.bucket[t];
      rank[j] = atomicAdd(&h[bk[j]], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSchedBuckets; i += blockDim.x)
    start[i] = h[i] ? atomicAdd(&s.cursor[i], h[i]) : 0u;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const long long t = base + (long long)j * kSortBlock + threadIdx.x;
    if (bk[j] >= 0) {
      const unsigned int pos = start[bk[j]] + rank[j];
      if (pos < (unsigned long long)s.n) s.perm[pos] = (unsigned int)t;
    }
  }
}

}  // namespace

cudaError_t launch_sched(const SchedParams& s, cudaStream_t st) {
  if (s.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(s.hist, 0, kSchedBuckets * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  const long long per = (long long)kSortBlock * kPerThread;
  const unsigned grid = (unsigned)((s.n + per - 1) / per);
  sched_hist<<<grid, kSortBlock, 0, st>>>(s);
  sched_scan<<<1, kSchedBuckets, 0, st>>>(s);
  sched_scatter<<<grid, kSortBlock, 0, st>>>(s);
  return cudaGetLastError();
}

}  // namespace dg
