// Wide multitask network (the PyTorch network of the Multitasking model,
// Sec. 5): stimulus and task inputs (clamped) -> hidden (H logistic units,
// H = 64..256) -> response (16 logistic units), every unit time-averaging,
//   s <- (1 - rate) s + rate net + noise eps,  y = 1 / (1 + exp(-gain (s + bias))),
// synchronous update (Sec. 3.3), stop when the largest response exceeds the
// second largest by more than the threshold, or at max_steps.
// Noise of unit u (hidden 0..H-1, then response H..H+15) at step j is normal
// (j-1)(H+16) + u of the trial's stream.
//
// A CTA holds 128 trials (one M = 128 MMA tile) with four threads per trial:
// thread (row r, quarter q) keeps the integrator state of hidden units
// [q H/4, (q+1) H/4) of trial r in registers. The hidden net input is constant
// per trial (inputs are clamped); it is computed once per trial and kept in
// tensor memory (TMEM lane r). Per step:
//   1. every thread integrates its hidden units (reading y(t-1) first) and
//      writes y(t-1) into a shared-memory A tile as a bfloat16 hi + lo pair
//      (y = hi + lo to about 2^-17), K-major canonical layout;
//   2. one thread issues tcgen05.mma (kind::f16, M128 N16, K16 at a time) over
//      K = 2H: D[r][n] = sum_h (hi + lo)[r][h] W[n][h], accumulated in FP32 in
//      TMEM; the BF16 response weights (B operand) were staged into shared
//      memory once per CTA by a bulk (TMA) copy;
//   3. the quarter-0 threads read their row of D back (tcgen05.ld), integrate
//      the 16 response units and apply the stop rule; finished trials are
//      replaced from the global trial cursor.
// Every wait on an mbarrier is bounded by a clock limit; on expiry the kernel
// records the failure in a status word and leaves.
//
// TC = false is the CUDA-core comparison form: the same CTA layout, with the
// response net input summed from per-quarter partial dot products in shared
// memory instead of the tensor-core GEMM.
#include <cuda_bf16.h>

#include "dg_device.cuh"
#include "dg_internal.h"
#include "dg_tc.cuh"

namespace dg {

namespace {

constexpr int kRows = 128;        // trials per CTA
constexpr int kThreads = 512;     // four threads per trial
constexpr int kR = 16;            // response units

// ------------------------------------------------------------- layout ---

// Byte offset of the 8-element K run starting at kk (multiple of 8) in row
// `row` of a K-major canonical tile with `kdim` columns.
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int kk, int kdim) {
  return (uint32_t)(((row >> 3) * (kdim >> 3) + (kk >> 3)) * 128 + (row & 7) * 16);
}

template <int H, bool TC>
struct Lay {
  static constexpr int HQ = H / 4;      // hidden units per thread
  static constexpr int K2 = 2 * H;      // hi and lo halves along K
  static constexpr int U = H + kR;      // noisy units
  // TC: B tile (BF16 [16][K2]) + A tile (BF16 [128][K2]); plain: FP32 W [16][H] +
  // partial sums [4][16][128] + hidden net [H][128]
  static constexpr uint32_t B_OFF = 0;
  static constexpr uint32_t B_BYTES = TC ? kR * K2 * 2 : kR * H * 4;
  static constexpr uint32_t A_OFF = (B_BYTES + 1023) / 1024 * 1024;
  static constexpr uint32_t A_BYTES = TC ? kRows * K2 * 2 : (4 * kR * kRows + H * kRows) * 4;
  static constexpr uint32_t WIN_OFF = A_OFF + A_BYTES;
};

struct WideShared {
  uint64_t bar_load;
  uint64_t bar_mma;
  uint32_t tmem_base;
  int fail;
  long long slot[kRows];
  float yr[kR][kRows];   // response outputs of the step, [unit][trial row]
};

// y = hi + lo with hi = bf16(y), lo = bf16(y - hi); two values per word, one
// paired conversion for each half.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int H, bool TC>
__global__ void __launch_bounds__(kThreads, 1) wide_kernel(WideParams p) {
  using L = Lay<H, TC>;
  constexpr int HQ = L::HQ, NCH = HQ / 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ WideShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp >> 2;                   // quarter of the hidden units
  const int r = ((warp & 3) << 5) | lane;    // trial row = TMEM lane
  const int nin = p.S + p.T;
  float* w_in = reinterpret_cast<float*>(smem + L::WIN_OFF);   // [H][nin]

  // ---- set-up: TMEM, barriers, weights staged by bulk copies
  if (TC && warp == 0) {
    tmem_alloc(&sh.tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&sh.bar_load, 1);
    mbar_init(&sh.bar_mma, 1);
    fence_mbar_init();
    sh.fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    const uint32_t wb = L::B_BYTES, ib = (uint32_t)(H * nin * 4);
    mbar_expect_tx(&sh.bar_load, wb + ib);
    bulk_g2s(smem + L::B_OFF, TC ? (const void*)p.w_resp_bf16 : (const void*)p.w_resp_f32, wb,
             &sh.bar_load);
    bulk_g2s(w_in, p.w_in, ib, &sh.bar_load);
  }
  if (!mbar_wait(&sh.bar_load, 0)) {
    atomicExch(p.status, 1);
    sh.fail = 1;
  }
  const uint32_t tmem = TC ? sh.tmem_base : 0u;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;   // this warp's TMEM lanes
  const uint32_t tmem_d = tmem + 256u;                            // accumulator columns

  // ---- first trials
  if (q == 0) {
    const long long f = fetch_trial(p.cursor, true);
    sh.slot[r] = (f >= 0 && f < p.n) ? f : -1;
  }
  __syncthreads();

  float s[HQ];
  float sr[4];        // response units 4q .. 4q+3 of this thread's trial
  long long t = -1;
  int k = 0;
  uint32_t phase = 0;
  const float keep = 1.0f - p.rate;
  const Logistic lg_h = Logistic::of(p.gain_h, p.bias_h), lg_r = Logistic::of(p.gain_r, p.bias_r);
  float* net_sm = reinterpret_cast<float*>(smem + L::A_OFF) + 4 * kR * kRows;  // plain: [H][128]
  float* part = reinterpret_cast<float*>(smem + L::A_OFF);                      // plain: [4][16][128]

  while (true) {
    // ---- (re)start trials whose slot changed
    const long long ns = sh.slot[r];
    const bool fresh = ns != t;
    t = ns;
    if (fresh) {
      k = 0;
#pragma unroll
      for (int i = 0; i < HQ; ++i) s[i] = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) sr[i] = 0.f;
    }
    const bool active = t >= 0;
    if (__any_sync(kFull, fresh)) {
      // hidden net input of the new trial, once: net_h = sum_q W_in[h][q] c[q]
      const float* cin = p.cond;
      if (active) {
        const long long g = (long long)p.trial0 + t;
        cin = p.cond + (size_t)((g / p.cond_block) % p.n_cond) * nin;
      }
#pragma unroll 1
      for (int c = 0; c < NCH; ++c) {
        float nv[16];
        if (TC) tmem_ld16(tmem + lane_base + (uint32_t)(q * HQ + 16 * c), nv);
        if (fresh && active) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float* w = w_in + (size_t)(q * HQ + 16 * c + i) * nin;
            float acc = 0.f;
            for (int j = 0; j < nin; ++j) acc = fmaf(w[j], __ldg(cin + j), acc);
            nv[i] = acc;
          }
        }
        if (TC) {
          tmem_st16(tmem + lane_base + (uint32_t)(q * HQ + 16 * c), nv);
        } else if (fresh && active) {
#pragma unroll
          for (int i = 0; i < 16; ++i) net_sm[(q * HQ + 16 * c + i) * kRows + r] = nv[i];
        }
      }
    }
    if (!__syncthreads_or(active ? 1 : 0) || sh.fail) break;

    // ---- 1. hidden units: read y(t-1), integrate, publish y(t-1)
    const uint32_t tg = p.trial0 + (uint32_t)(active ? t : 0);
    const uint32_t blk0 = (uint32_t)k * (uint32_t)(L::U / 4) + (uint32_t)(q * (HQ / 4));
    float acc[kR];
#pragma unroll
    for (int n = 0; n < kR; ++n) acc[n] = 0.f;
    // eight hidden units (two Philox blocks) at a time; a warp whose 32 rows
    // hold no running trial skips the work (its rows of D are not read)
    const bool warp_live = __any_sync(kFull, active);
#pragma unroll
    for (int c = 0; c < HQ / 8; ++c) {
      if (!warp_live) break;
      float nv[8];
      if (TC) {
        tmem_ld8(tmem + lane_base + (uint32_t)(q * HQ + 8 * c), nv);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) nv[i] = net_sm[(q * HQ + 8 * c + i) * kRows + r];
      }
      float e[8];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float4 z = normals4(noise_block_rk(p.rk, tg, 0u, blk0 + (uint32_t)(2 * c + b)));
        e[4 * b] = z.x;
        e[4 * b + 1] = z.y;
        e[4 * b + 2] = z.z;
        e[4 * b + 3] = z.w;
      }
      float y[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float& sv = s[8 * c + i];
        y[i] = lg_h(sv);
        sv = fmaf(keep, sv, fmaf(p.rate, nv[i], p.noise * e[i]));
      }
      if (TC) {
        unsigned char* A = smem + L::A_OFF;
        const int kk = q * HQ + 8 * c;
        uint4 hi, lo;
        split2(y[0], y[1], hi.x, lo.x);
        split2(y[2], y[3], hi.y, lo.y);
        split2(y[4], y[5], hi.z, lo.z);
        split2(y[6], y[7], hi.w, lo.w);
        *reinterpret_cast<uint4*>(A + kmajor_off(r, kk, L::K2)) = hi;
        *reinterpret_cast<uint4*>(A + kmajor_off(r, H + kk, L::K2)) = lo;
      } else {
        const float* W = reinterpret_cast<const float*>(smem + L::B_OFF);   // [16][H]
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int h = q * HQ + 8 * c + i;
#pragma unroll
          for (int n = 0; n < kR; ++n) acc[n] = fmaf(W[n * H + h], y[i], acc[n]);
        }
      }
    }
    if (TC) {
      fence_proxy_async();
      tc_fence_before();
    } else {
#pragma unroll
      for (int n = 0; n < kR; ++n) part[(q * kR + n) * kRows + r] = acc[n];
    }
    __syncthreads();

    // ---- 2. response net input D = y(t-1) W^T on the tensor cores
    if (TC && tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem + L::A_OFF), b0 = smem_u32(smem + L::B_OFF);
      const uint32_t sbo = (uint32_t)(L::K2 / 8) * 128u;
      constexpr uint32_t idesc = mma_idesc(kRows, kR);
#pragma unroll 1
      for (int kc = 0; kc < L::K2 / 16; ++kc) {
        const uint32_t off = (uint32_t)kc * 256u;   // two core matrices along K
        mma_bf16(tmem_d, smem_desc(a0 + off, 128u, sbo), smem_desc(b0 + off, 128u, sbo), idesc,
                 kc > 0 ? 1u : 0u);
      }
      mma_commit(&sh.bar_mma);
    }

    // ---- 3. response units 4q .. 4q+3 of every trial (all quarters); their
    // normals do not depend on D, so they are drawn while the MMA runs
    {
      float4 zr = make_float4(0.f, 0.f, 0.f, 0.f);
      if (warp_live)
        zr = normals4(noise_block_rk(
            p.rk, tg, 0u, (uint32_t)k * (uint32_t)(L::U / 4) + (uint32_t)(H / 4 + q)));
      float net[4];
      if (TC) {
        if (!mbar_wait(&sh.bar_mma, phase)) {
          atomicExch(p.status, 1);
          sh.fail = 1;
        }
        tc_fence_after();
        tmem_ld4(tmem_d + lane_base + (uint32_t)(4 * q), net);
        tc_fence_before();
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = 4 * q + j;
          net[j] = ((part[(0 * kR + n) * kRows + r] + part[(1 * kR + n) * kRows + r]) +
                    part[(2 * kR + n) * kRows + r]) + part[(3 * kR + n) * kRows + r];
        }
      }
      if (warp_live) {
        const float e4[4] = {zr.x, zr.y, zr.z, zr.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          sr[j] = fmaf(keep, sr[j], fmaf(p.rate, net[j], p.noise * e4[j]));
          sh.yr[4 * q + j][r] = lg_r(sr[j]);
        }
      }
    }
    phase ^= 1u;
    __syncthreads();

    // ---- stop rule on the 16 responses; refill finished rows (quarter 0)
    if (q == 0) {
      bool finished = false;
      if (active) {
        int best = 0;
        float v1 = sh.yr[0][r];
#pragma unroll
        for (int n = 1; n < kR; ++n) {
          const float v = sh.yr[n][r];
          if (v > v1) {
            v1 = v;
            best = n;
          }
        }
        float v2 = -INFINITY;
#pragma unroll
        for (int n = 0; n < kR; ++n)
          if (n != best) v2 = fmaxf(v2, sh.yr[n][r]);
        const bool hit = v1 - v2 > p.stop_threshold;
        if (hit || k + 1 >= p.max_steps) {
          p.choice[t] = hit ? (int8_t)best : (int8_t)-1;
          p.step[t] = hit ? k + 1 : p.max_steps;
          if (p.yout)
#pragma unroll
            for (int n = 0; n < kR; ++n) p.yout[(size_t)t * kR + n] = sh.yr[n][r];
          finished = true;
        }
      }
      const long long f = fetch_trial(p.cursor, finished);
      if (finished) sh.slot[r] = (f >= 0 && f < p.n) ? f : -1;
    }
    ++k;
    __syncthreads();
  }

  // ---- tear-down
  __syncthreads();
  if (TC) {
    if (sh.fail) {
      // give an MMA that may still be in flight a bounded time to finish
      if (tid == 0) mbar_wait(&sh.bar_mma, phase ^ 1u);
      __syncthreads();
    }
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
  }
}

template <int H, bool TC>
cudaError_t launch_h(const WideParams& p, cudaStream_t s) {
  using L = Lay<H, TC>;
  size_t smem = L::WIN_OFF + (size_t)H * (p.S + p.T) * 4;
  // more than half of an SM's shared memory, so that two CTAs never share an
  // SM (each takes all 512 TMEM columns)
  if (smem < 120 * 1024) smem = 120 * 1024;
  cudaError_t e = smem_limit((const void*)wide_kernel<H, TC>, (int)smem);
  if (e != cudaSuccess) return e;
  long long grid = (p.n + kRows - 1) / kRows;
  const long long cap = (long long)num_sms();  // one CTA per SM (all of its TMEM)
  if (grid > cap) grid = cap;
  wide_kernel<H, TC><<<(unsigned)grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t wide_smem_bytes(int H, int nin, bool tc) {
  const size_t b = tc ? (size_t)kR * 2 * H * 2 : (size_t)kR * H * 4;
  const size_t a_off = (b + 1023) / 1024 * 1024;
  const size_t a = tc ? (size_t)kRows * 2 * H * 2 : (size_t)(4 * kR * kRows + H * kRows) * 4;
  return a_off + a + (size_t)H * nin * 4;
}

void wide_b_image(const uint16_t* w_bf16, int H, uint16_t* img) {
  // B operand image: row n of K2 = 2H elements is [W[n][0..H) | W[n][0..H)],
  // in the K-major canonical layout of the tensor-core tile
  const int K2 = 2 * H;
  for (int n = 0; n < kR; ++n)
    for (int kk = 0; kk < K2; kk += 8) {
      const uint32_t off = kmajor_off(n, kk, K2) / 2;
      for (int j = 0; j < 8; ++j) img[off + j] = w_bf16[(size_t)n * H + ((kk + j) % H)];
    }
}

cudaError_t launch_wide(const WideParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  (void)cfg;
  if (p.n <= 0) return cudaSuccess;
  const bool tc = mode == 0;
  switch (p.H) {
    case 64: return tc ? launch_h<64, true>(p, s) : launch_h<64, false>(p, s);
    case 128: return tc ? launch_h<128, true>(p, s) : launch_h<128, false>(p, s);
    case 192: return tc ? launch_h<192, true>(p, s) : launch_h<192, false>(p, s);
    case 256: return tc ? launch_h<256, true>(p, s) : launch_h<256, false>(p, s);
  }
  return cudaErrorNotSupported;
}

}  // namespace dg
