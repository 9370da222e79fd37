// Leaky competing accumulator trials (Sec. 4.4, the LCA of the Multitasking
// model in Sec. 5), Usher-McClelland form, synchronous update:
//   x_i <- x_i + ((I_i - k x_i - beta sum_{j != i} x_j) dt + sigma sqrt(dt) eps_i)
//   x_i <- max(0, x_i)                         (unless DG_LCA_NO_RECTIFY)
// evaluated as x_i <- x_i + (g x_i + (dt I_i - c S) + sigma sqrt(dt) eps_i) with
// S = sum_j x_j, g = dt (beta - k), c = dt beta: the same update in five
// instructions per accumulator (dt I_i is formed once per trial). The
// increment is formed apart from x_i: folding 1 + g into one coefficient
// would round it once and compound that error over thousands of steps.
// stop when max_i x_i >= threshold (winner = lowest index among maxima), or,
// two-sided with N = 1, when |x| >= threshold (the DDM mapping of Sec. 4.4).
// eps_i of step j (1-based) is normal (j-1) N + i of the (seed, trial, 0) stream.
//
// A trial is held by a group of TPT lanes (threads per trial), each holding
// N / TPT accumulators in registers; the sum and the max go through shuffles
// inside the group. Batched form: persistent grid, groups refill from a global
// trial cursor. Plain form: one thread per trial, one launch.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

template <int N, int TPT>
struct Lca {
  static constexpr int NU = N / TPT;  // accumulators per lane

  // Normals of this lane's units for step index k (0-based).
  static __device__ __forceinline__ void noise(const LcaParams& p, uint32_t trial, int k, int g,
                                               float (&e)[NU]) {
    noise_k(p.rk, trial, k, g, e);
  }

  template <typename Keys>
  static __device__ __forceinline__ void noise_k(const Keys& rk, uint32_t trial, int k, int g,
                                                 float (&e)[NU]) {
    if constexpr (NU % 4 == 0) {
      const uint32_t b0 = (uint32_t)k * (uint32_t)(N / 4) + (uint32_t)(g * (NU / 4));
#pragma unroll
      for (int b = 0; b < NU / 4; ++b) {
        const float4 z = normals4(noise_block_rk(rk, trial, 0u, b0 + (uint32_t)b));
        e[4 * b + 0] = z.x;
        e[4 * b + 1] = z.y;
        e[4 * b + 2] = z.z;
        e[4 * b + 3] = z.w;
      }
    } else {
      static_assert(TPT == 1, "split trials need whole Philox blocks per lane");
      const uint32_t d0 = (uint32_t)k * (uint32_t)N;
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        const uint32_t d = d0 + (uint32_t)i;
        if (i == 0 || (d & 3u) == 0u) z = normals4(noise_block_rk(rk, trial, 0u, d >> 2));
        e[i] = pick4(z, d & 3u);
      }
    }
  }

  // S = sum of the N accumulators in one fixed order for every layout: a
  // balanced pairwise tree over units in index order when N is a power of
  // two (each lane reduces its contiguous chunk, then lanes combine with
  // ascending shuffle distances, which continues the same tree), else a
  // sequential sum (those N run with one lane per trial only).
  static __device__ __forceinline__ float chunk_sum(const float (&x)[NU]) {
    if constexpr ((N & (N - 1)) == 0) {
      float t[NU];
#pragma unroll
      for (int i = 0; i < NU; ++i) t[i] = x[i];
#pragma unroll
      for (int w = 1; w < NU; w <<= 1)
#pragma unroll
        for (int i = 0; i + w < NU; i += 2 * w) t[i] = t[i] + t[i + w];
      return t[0];
    } else {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < NU; ++i) s += x[i];
      return s;
    }
  }

  static __device__ __forceinline__ float group_sum(float v, unsigned gmask) {
#pragma unroll
    for (int o = 1; o < TPT; o <<= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
  }

  static __device__ __forceinline__ float group_max(float v, unsigned gmask) {
#pragma unroll
    for (int o = TPT / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(gmask, v, o));
    return v;
  }

  static __device__ __forceinline__ int group_min(int v, unsigned gmask) {
#pragma unroll
    for (int o = TPT / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(gmask, v, o));
    return v;
  }

  // One step of one trial with its normals e; I holds dt I_i. Returns true
  // when the trial has ended at this step.
  static __device__ __forceinline__ bool step(const LcaParams& p, const float (&e)[NU], int g,
                                              unsigned gmask, float (&x)[NU], const float (&I)[NU],
                                              int8_t& choice) {
    const float S = group_sum(chunk_sum(x), gmask);
    // every multiply-add written as fmaf, so that each layout and form
    // computes the same bits (no contraction left to the compiler)
    const float gr = p.dt * (p.inhibition - p.leak);   // g
    const float c = p.dt * p.inhibition;
    // with eight or more accumulators per lane, adjacent ones by the paired
    // FP32 instructions (each component rounded as the scalar fmaf and add;
    // measured faster at N = 8, slower at N = 4); the rest one at a time
    constexpr int NP = NU >= 8 ? NU / 2 * 2 : 0;   // accumulators taken in pairs
#pragma unroll
    for (int i = 0; i + 1 < NP; i += 2) {
      const float2 xi = make_float2(x[i], x[i + 1]);
      float2 v = __ffma2_rn(make_float2(-c, -c), make_float2(S, S), make_float2(I[i], I[i + 1]));
      v = __ffma2_rn(make_float2(p.diffusion, p.diffusion), make_float2(e[i], e[i + 1]), v);
      v = __fadd2_rn(xi, __ffma2_rn(make_float2(gr, gr), xi, v));
      if (p.rectify) {
        v.x = fmaxf(v.x, 0.f);
        v.y = fmaxf(v.y, 0.f);
      }
      x[i] = v.x;
      x[i + 1] = v.y;
    }
#pragma unroll
    for (int i = NP; i < NU; ++i) {
      float v = x[i] + fmaf(gr, x[i], fmaf(p.diffusion, e[i], fmaf(-c, S, I[i])));
      if (p.rectify) v = fmaxf(v, 0.f);
      x[i] = v;
    }
    if (N == 1 && p.two_sided) {
      if (fabsf(x[0]) >= p.threshold) {
        choice = x[0] > 0.f ? 1 : 0;
        return true;
      }
      return false;
    }
    // the stop test needs only the largest state; the winner (the lowest
    // index holding it) is looked up on the step that reaches the threshold
    float m = x[0];
#pragma unroll
    for (int i = 1; i < NU; ++i) m = fmaxf(m, x[i]);
    m = group_max(m, gmask);
    if (m >= p.threshold) {
      int mi = N;
#pragma unroll
      for (int i = NU - 1; i >= 0; --i)
        if (x[i] == m) mi = g * NU + i;
      choice = (int8_t)group_min(mi, gmask);
      return true;
    }
    return false;
  }

  static __device__ __forceinline__ void load(const LcaParams& p, long long t, int g,
                                              float (&x)[NU], float (&I)[NU]) {
    const float* src = p.I + (size_t)t * N + g * NU;
#pragma unroll
    for (int i = 0; i < NU; ++i) {
      I[i] = p.dt * __ldg(src + i);   // dt I_i
      x[i] = 0.f;
    }
  }

  static __device__ __forceinline__ void store(const LcaParams& p, long long t, int g, int8_t c,
                                               int st, const float (&x)[NU]) {
    if (g == 0) {
      p.choice[t] = c;
      p.step[t] = st;
    }
    if (p.xout) {
      float* dst = p.xout + (size_t)t * N + g * NU;
#pragma unroll
      for (int i = 0; i < NU; ++i) dst[i] = x[i];
    }
  }
};

template <int N, int TPT>
__global__ void __launch_bounds__(256) lca_batched(LcaParams p) {
  using L = Lca<N, TPT>;
  const int lane = threadIdx.x & 31;
  const int g = lane % TPT;
  const int root = lane - g;
  const unsigned gmask = (TPT == 32 ? kFull : ((1u << TPT) - 1u)) << root;
  float x[L::NU], I[L::NU], e[L::NU];
  long long f = fetch_trial(p.cursor, g == 0);
  f = __shfl_sync(kFull, f, root);
  bool active = f >= 0 && f < p.n;
  long long t = active ? (p.perm ? (long long)__ldg(p.perm + f) : f) : 0;
  int k = 0;
  if (active) {
    L::load(p, t, g, x, I);
    L::noise(p, p.trial0 + (uint32_t)t, 0, g, e);
  }
  while (__any_sync(kFull, active)) {
    bool finished = false;
    if (active) {
      // the next step's normals do not depend on the state: drawn alongside
      // this step's update, they take the noise off the step's critical path
      float en[L::NU];
      L::noise(p, p.trial0 + (uint32_t)t, k + 1, g, en);
      int8_t c = -1;
      const bool hit = L::step(p, e, g, gmask, x, I, c);
      ++k;
      if (hit || k >= p.max_steps) {
        L::store(p, t, g, hit ? c : (int8_t)-1, hit ? k : p.max_steps, x);
        finished = true;
      }
#pragma unroll
      for (int i = 0; i < L::NU; ++i) e[i] = en[i];
    }
    f = fetch_trial(p.cursor, finished && g == 0);
    f = __shfl_sync(kFull, f, root);
    if (finished) {
      active = f < p.n;
      k = 0;
      if (active) {
        t = p.perm ? (long long)__ldg(p.perm + f) : f;
        L::load(p, t, g, x, I);
        L::noise(p, p.trial0 + (uint32_t)t, 0, g, e);
      }
    }
  }
}

// Batched form with block-level compaction (one lane per trial). With about
// as many lanes as trials every trial starts at once and a warp would run
// until its slowest lane ends. Here the block runs in chunks of p.chunk steps;
// after each chunk the trials still running are packed into the block's
// leading lanes through shared memory (trial, step, state, next noise), the
// freed lanes take new trials from the cursor, and warps left without a trial
// sit out the next chunk. Lanes change trials, never results.
// Shared memory of lca_compact<N>: x, I and next-step noise per lane, trial and step.
inline size_t compact_smem(int N) { return (3 * (size_t)N * 256) * sizeof(float) + 256 * (8 + 4); }

// The rest of one trial on a whole warp (N a multiple of 4): the lanes draw
// the noise of 32 / (N / 4) steps at once (lane l: Philox block l mod N/4 of
// step k + l div (N/4)), then every lane takes those steps on its own copy of
// the state, gathering each step's normals by shuffles. The arithmetic is the
// one-lane step's, so the trial ends exactly as it would have.
template <int N, typename Keys>
__device__ void lca_warp_trial(const LcaParams& p, const Keys& rk, long long t, int k,
                               float (&x)[N], const float (&I)[N]) {
  using L = Lca<N, 1>;
  constexpr int NB = N / 4, R = 32 / NB;
  const int lane = threadIdx.x & 31;
  const uint32_t trial = p.trial0 + (uint32_t)t;
  while (true) {
    const float4 z = normals4(noise_block_rk(
        rk, trial, 0u, (uint32_t)(k + lane / NB) * (uint32_t)NB + (uint32_t)(lane % NB)));
#pragma unroll 1
    for (int s = 0; s < R; ++s) {
      float e[N];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int src = s * NB + b;
        e[4 * b] = __shfl_sync(kFull, z.x, src);
        e[4 * b + 1] = __shfl_sync(kFull, z.y, src);
        e[4 * b + 2] = __shfl_sync(kFull, z.z, src);
        e[4 * b + 3] = __shfl_sync(kFull, z.w, src);
      }
      int8_t c = -1;
      const bool hit = L::step(p, e, 0, kFull, x, I, c);
      ++k;
      if (hit || k >= p.max_steps) {
        if (lane == 0) L::store(p, t, 0, hit ? c : (int8_t)-1, hit ? k : p.max_steps, x);
        return;
      }
    }
  }
}

// MULTI: the trials of several jobs of one model (the serving loop's groups),
// one list over the jobs in order; a lane holds its trial's list index f and
// binds the trial's job (inputs, outputs, seed, trial offset) when it takes
// the trial on, so a trial ends exactly as in a launch of its job alone.
template <int N, bool MULTI>
__global__ void __launch_bounds__(256) lca_compact(
    LcaParams p, const __grid_constant__ typename TableOf<MULTI>::type tab) {
  using L = Lca<N, 1>;
  extern __shared__ __align__(16) float csm[];
  float* s_x = csm;                          // [N][256]
  float* s_I = csm + N * 256;                // [N][256]
  float* s_e = csm + 2 * N * 256;            // [N][256]
  long long* s_t = reinterpret_cast<long long*>(csm + 3 * N * 256);   // [256]
  int* s_k = reinterpret_cast<int*>(s_t + 256);                        // [256]
  __shared__ int warp_cnt[8];
  __shared__ MultiJob s_job[MULTI ? kMaxMultiJobs : 1];
  if constexpr (MULTI) copy_jobs(tab, s_job);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned self = 1u << lane;
  float x[N], I[N], e[N];
  // the lane's trial: t its index in its job, f its list entry (MULTI), q the
  // launch's parameters with the job's inputs, outputs and trial offset
  LcaParams q = p;
  KeyPair kp{};
  long long t = 0, f = 0;
  int k = 0;
  auto bind = [&](long long fi) {
    if constexpr (MULTI) {
      const MultiJob& J = s_job[multi_job_of(s_job, tab.n_jobs, fi)];
      q.I = J.in;
      q.choice = J.choice;
      q.step = J.step;
      q.xout = J.xout;
      q.trial0 = J.trial0;
      kp.k.k0 = J.k0;
      kp.k.k1 = J.k1;
      f = fi;
      t = fi - J.start;
    } else {
      t = p.perm ? (long long)__ldg(p.perm + fi) : fi;
    }
  };
  auto noise = [&](int kk, float (&out)[N]) {
    if constexpr (MULTI)
      L::noise_k(kp, q.trial0 + (uint32_t)t, kk, 0, out);
    else
      L::noise(p, p.trial0 + (uint32_t)t, kk, 0, out);
  };
  long long fc = fetch_trial(p.cursor, true);
  bool active = fc >= 0 && fc < p.n;
  if (active) {
    bind(fc);
    L::load(q, t, 0, x, I);
    noise(0, e);
  }
  while (true) {
    // ---- a chunk of steps
    // (N >= 8, one job: two steps per iteration, the noise buffers in turn: the second
    // step draws the step after it into e, so no copy is made, and a chunk of
    // p.chunk steps rounds up to an even count; for smaller N the second copy
    // of the step costs more in occupancy than it saves)
    constexpr int kPer = N >= 8 && !MULTI ? 2 : 1;
    if (__any_sync(kFull, active)) {
      for (int s = 0; s < p.chunk; s += kPer) {
        if (kPer == 1 && active) {
          float en[N];
          noise(k + 1, en);
          int8_t c = -1;
          const bool hit = L::step(p, e, 0, self, x, I, c);
          ++k;
          if (hit || k >= p.max_steps) {
            L::store(q, t, 0, hit ? c : (int8_t)-1, hit ? k : p.max_steps, x);
            active = false;
          }
#pragma unroll
          for (int i = 0; i < N; ++i) e[i] = en[i];
        } else if (kPer == 2 && active) {
          float en[N];
          noise(k + 1, en);
          int8_t c = -1;
          bool hit = L::step(p, e, 0, self, x, I, c);
          ++k;
          if (hit || k >= p.max_steps) {
            L::store(q, t, 0, hit ? c : (int8_t)-1, hit ? k : p.max_steps, x);
            active = false;
          } else {
            noise(k + 1, e);
            c = -1;
            hit = L::step(p, en, 0, self, x, I, c);
            ++k;
            if (hit || k >= p.max_steps) {
              L::store(q, t, 0, hit ? c : (int8_t)-1, hit ? k : p.max_steps, x);
              active = false;
            }
          }
        }
        if (!__any_sync(kFull, active)) break;
      }
    }
    // ---- pack the running trials into the leading lanes
    const unsigned live = __ballot_sync(kFull, active);
    if (lane == 0) warp_cnt[warp] = __popc(live);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int c = warp_cnt[w];
      if (w < warp) before += c;
      total += c;
    }
    if (active) {
      const int d = before + __popc(live & (self - 1u));
#pragma unroll
      for (int i = 0; i < N; ++i) {
        s_x[i * 256 + d] = x[i];
        s_I[i * 256 + d] = I[i];
        s_e[i * 256 + d] = e[i];
      }
      s_t[d] = MULTI ? f : t;
      s_k[d] = k;
    }
    __syncthreads();
    active = tid < total;
    if (active) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        x[i] = s_x[i * 256 + tid];
        I[i] = s_I[i * 256 + tid];
        e[i] = s_e[i * 256 + tid];
      }
      if constexpr (MULTI)
        bind(s_t[tid]);
      else
        t = s_t[tid];
      k = s_k[tid];
    }
    // ---- the free lanes take new trials
    fc = fetch_trial(p.cursor, !active);
    const bool refilled = !active && fc >= 0 && fc < p.n;
    if (refilled) {
      active = true;
      bind(fc);
      k = 0;
      L::load(q, t, 0, x, I);
      noise(0, e);
    }
    if constexpr (N % 4 == 0) {
      // no trial left to hand out and at most one per warp still running: a
      // warp each, so that the last, longest trials run at a warp's pace
      if (!__syncthreads_or(refilled ? 1 : 0) && total > 0 && total <= p.tail_max) {
        if (warp < total) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            x[i] = s_x[i * 256 + warp];
            I[i] = s_I[i * 256 + warp];
          }
          if constexpr (MULTI) {
            bind(s_t[warp]);
            lca_warp_trial<N>(q, kp, t, s_k[warp], x, I);
          } else {
            lca_warp_trial<N>(p, p.rk, s_t[warp], s_k[warp], x, I);
          }
        }
        return;
      }
    }
    if (!__syncthreads_or(active ? 1 : 0)) break;
  }
}

template <int N>
__global__ void __launch_bounds__(256) lca_plain(LcaParams p) {
  using L = Lca<N, 1>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = 1u << lane;
  float x[L::NU], I[L::NU];
  L::load(p, t, 0, x, I);
  for (int k = 0; k < p.max_steps; ++k) {
    int8_t c = -1;
    float e[L::NU];
    L::noise(p, p.trial0 + (uint32_t)t, k, 0, e);
    if (L::step(p, e, 0, gmask, x, I, c)) {
      L::store(p, t, 0, c, k + 1, x);
      return;
    }
  }
  L::store(p, t, 0, (int8_t)-1, p.max_steps, x);
}

template <int N, int TPT>
void* batched_fn() {
  return (void*)lca_batched<N, TPT>;
}

template <int N>
cudaError_t launch_n(const LcaParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  if (mode == 1) {
    const int block = 256;
    const long long grid = (p.n + block - 1) / block;
    lca_plain<N><<<(unsigned)grid, block, 0, s>>>(p);
    return cudaGetLastError();
  }
  const int block = cfg.block;
  int grid = cfg.grid;
  if (grid <= 0) grid = num_sms() * lca_max_blocks_per_sm(N, cfg.tpt, block);
  const long long need = (p.n * (cfg.tpt > 0 ? cfg.tpt : 1) + block - 1) / block;
  if (grid > need) grid = (int)need;
  if (grid < 1) grid = 1;
  switch (cfg.tpt) {
    case 0: {   // block-level compaction, one lane per trial (256 threads)
      if constexpr (N <= 16) {
        const size_t smem = compact_smem(N);
        const cudaError_t ea = smem_limit((const void*)lca_compact<N, false>, (int)smem);
        if (ea != cudaSuccess) return ea;
        lca_compact<N, false><<<grid, 256, smem, s>>>(p, {});
        break;
      }
      return cudaErrorInvalidValue;
    }
    case 1: lca_batched<N, 1><<<grid, block, 0, s>>>(p); break;
    case 2:
      if constexpr (N % 8 == 0) { lca_batched<N, 2><<<grid, block, 0, s>>>(p); break; }
      return cudaErrorInvalidValue;
    case 4:
      if constexpr (N % 16 == 0) { lca_batched<N, 4><<<grid, block, 0, s>>>(p); break; }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_multi_n(const LcaParams& p, const MultiJobTable& tab, cudaStream_t s) {
  const size_t smem = compact_smem(N);
  const void* fn = (const void*)lca_compact<N, true>;
  cudaError_t e = smem_limit(fn, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, smem)) != cudaSuccess)
    return e;
  long long grid = (long long)num_sms() * (nb > 0 ? nb : 1);
  const long long need = (p.n + 255) / 256;   // one lane per trial
  if (grid > need) grid = need;
  lca_compact<N, true><<<(unsigned)grid, 256, smem, s>>>(p, tab);
  return cudaGetLastError();
}

template <int N>
void* compact_fn() {
  return (void*)lca_compact<N, false>;
}

void* kernel_for(int N, int tpt) {
  switch (tpt) {
    case 0:
      switch (N) {
#define DG_CASE(n) case n: return compact_fn<n>();
        DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8)
        DG_CASE(9) DG_CASE(10) DG_CASE(11) DG_CASE(12) DG_CASE(13) DG_CASE(14) DG_CASE(15)
        DG_CASE(16)
#undef DG_CASE
      }
      return nullptr;
    case 1:
      switch (N) {
#define DG_CASE(n) case n: return batched_fn<n, 1>();
        DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8)
        DG_CASE(9) DG_CASE(10) DG_CASE(11) DG_CASE(12) DG_CASE(13) DG_CASE(14) DG_CASE(15)
        DG_CASE(16)
#undef DG_CASE
      }
      return nullptr;
    case 2:
      if (N == 8) return batched_fn<8, 2>();
      if (N == 16) return batched_fn<16, 2>();
      return nullptr;
    case 4:
      if (N == 16) return batched_fn<16, 4>();
      return nullptr;
  }
  return nullptr;
}

}  // namespace

cudaError_t launch_lca_multi(const LcaParams& p, const MultiJobTable& tab, cudaStream_t s) {
  if (p.n <= 0 || tab.n_jobs < 1 || tab.n_jobs > kMaxMultiJobs) return cudaErrorInvalidValue;
  switch (p.N) {
#define DG_CASE(n) case n: return launch_multi_n<n>(p, tab, s);
    DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8)
    DG_CASE(9) DG_CASE(10) DG_CASE(11) DG_CASE(12) DG_CASE(13) DG_CASE(14) DG_CASE(15)
    DG_CASE(16)
#undef DG_CASE
  }
  return cudaErrorInvalidValue;
}

bool lca_tpt_supported(int N, int tpt) { return kernel_for(N, tpt) != nullptr; }

int lca_max_blocks_per_sm(int N, int tpt, int block) {
  void* fn = kernel_for(N, tpt);
  if (!fn) return 0;
  int nb = 0;
  if (tpt == 0) {
    if (smem_limit(fn, (int)compact_smem(N)) != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, compact_smem(N));
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0);
  }
  return nb;
}

cudaError_t launch_lca(const LcaParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  switch (p.N) {
#define DG_CASE(n) case n: return launch_n<n>(p, mode, cfg, s);
    DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8)
    DG_CASE(9) DG_CASE(10) DG_CASE(11) DG_CASE(12) DG_CASE(13) DG_CASE(14) DG_CASE(15)
    DG_CASE(16)
#undef DG_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace dg
