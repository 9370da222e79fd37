// Wide multitask network (the PyTorch network of the Multitasking model,
// Sec. 5): stimulus and task inputs (clamped) -> hidden (H logistic units,
// H = 64..256) -> response (16 logistic units), every unit time-averaging,
//   s <- (1 - rate) s + rate net + noise eps,  y = 1 / (1 + exp(-gain (s + bias))),
// synchronous update (Sec. 3.3), stop when the largest response exceeds the
// second largest by more than the threshold, or at max_steps.
// Noise of unit u (hidden 0..H-1, then response H..H+15) at step j is normal
// (j-1)(H+16) + u of the trial's stream.
//
// Two forms:
//   - wide_block_kernel (batched form, tensor cores): trial slots advanced a
//     block of steps at a time, the response layer's inputs of all (step,
//     slot) rows of a block from one tcgen05.mma chain (described below);
//   - wide_rows_kernel (plain form, CUDA cores, the comparison form): a CTA
//     of 128 trial rows, four threads per trial, one step at a time, the
//     response net input summed from per-quarter partial dot products in
//     shared memory.
#include <cuda_bf16.h>

#include "dg_device.cuh"
#include "dg_internal.h"
#include "dg_tc.cuh"

namespace dg {

namespace {

constexpr int kRows = 128;        // trial rows of a CTA; rows of an MMA tile
constexpr int kR = 16;            // response units

// Byte offset of element (row, k) of a K-major bfloat16 tile of `rows` rows in
// the 128-byte swizzled layout of the tensor-core operands: K in atoms of 64
// elements (128 bytes per row), each atom holding all rows; rows in groups of
// eight (1024 bytes), and within a row the 16-byte chunk index XORed with the
// row's index in its group, so that eight rows' chunks fall in distinct banks.
__host__ __device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
  return (uint32_t)((k >> 6) * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((k & 63) >> 3) ^ (row & 7)) << 4) + (k & 7) * 2);
}

// y = hi + lo with hi = bf16(y), lo = bf16(y - hi) (y to about 2^-17); two
// values per word, one paired conversion for each half.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// ---------------------------------------------------------------------------
// Plain form on CUDA cores. Thread (row r, quarter q) keeps the states of
// hidden units [q H/4, (q+1) H/4) of trial r in registers; per step it
// integrates them, adds their products with the response weights into 16
// partial sums, and the quarter-0 threads integrate the response units from
// the four partial sums and apply the stop rule; finished rows take the next
// trial from the global cursor.

constexpr int kRowThreads = 512;  // four threads per trial row

template <int H>
struct RowLay {
  static constexpr int HQ = H / 4;      // hidden units per thread
  static constexpr int U = H + kR;      // noisy units
  // FP32 W [16][H], partial sums [4][16][128], hidden net [H][128], input weights [H][nin]
  static constexpr uint32_t W_OFF = 0;
  static constexpr uint32_t PART_OFF = (kR * H * 4 + 1023) / 1024 * 1024;
  static constexpr uint32_t NET_OFF = PART_OFF + 4 * kR * kRows * 4;
  static constexpr uint32_t WIN_OFF = NET_OFF + H * kRows * 4;
};

struct RowShared {
  uint64_t bar_load;
  int fail;
  long long slot[kRows];
  float yr[kR][kRows];   // response outputs of the step, [unit][trial row]
};

template <int H>
__global__ void __launch_bounds__(kRowThreads, 1) wide_rows_kernel(WideParams p) {
  using L = RowLay<H>;
  constexpr int HQ = L::HQ;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RowShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp >> 2;                   // quarter of the hidden units
  const int r = ((warp & 3) << 5) | lane;    // trial row
  const int nin = p.S + p.T;
  const float* W = reinterpret_cast<const float*>(smem + L::W_OFF);   // [16][H]
  float* part = reinterpret_cast<float*>(smem + L::PART_OFF);         // [4][16][128]
  float* net_sm = reinterpret_cast<float*>(smem + L::NET_OFF);        // [H][128]
  float* w_in = reinterpret_cast<float*>(smem + L::WIN_OFF);          // [H][nin]

  if (tid == 0) {
    mbar_init(&sh.bar_load, 1);
    fence_mbar_init();
    sh.fail = 0;
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t wb = kR * H * 4, ib = (uint32_t)(H * nin * 4);
    mbar_expect_tx(&sh.bar_load, wb + ib);
    bulk_g2s(smem + L::W_OFF, p.w_resp_f32, wb, &sh.bar_load);
    bulk_g2s(w_in, p.w_in, ib, &sh.bar_load);
  }
  if (!mbar_wait(&sh.bar_load, 0)) {
    atomicExch(p.status, 1);
    sh.fail = 1;
  }
  if (q == 0) {
    const long long f = fetch_trial(p.cursor, true);
    sh.slot[r] = (f >= 0 && f < p.n) ? f : -1;
  }
  __syncthreads();

  float s[HQ];
  float sr[4];        // response units 4q .. 4q+3 of this thread's trial
  long long t = -1;
  int k = 0;
  const float keep = 1.0f - p.rate;
  const Logistic lg_h = Logistic::of(p.gain_h, p.bias_h), lg_r = Logistic::of(p.gain_r, p.bias_r);

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
    if (fresh && active) {
      // hidden net input of the new trial, once: net_h = sum_j W_in[h][j] c[j]
      const long long g = (long long)p.trial0 + t;
      const float* cin = p.cond + (size_t)((g / p.cond_block) % p.n_cond) * nin;
#pragma unroll 1
      for (int i = 0; i < HQ; ++i) {
        const float* w = w_in + (size_t)(q * HQ + i) * nin;
        float acc = 0.f;
        for (int j = 0; j < nin; ++j) acc = fmaf(w[j], __ldg(cin + j), acc);
        net_sm[(q * HQ + i) * kRows + r] = acc;
      }
    }
    if (!__syncthreads_or(active ? 1 : 0) || sh.fail) break;

    // ---- hidden units: read y(t-1), integrate, add y(t-1) W^T into partial sums
    const uint32_t tg = p.trial0 + (uint32_t)(active ? t : 0);
    const uint32_t blk0 = (uint32_t)k * (uint32_t)(L::U / 4) + (uint32_t)(q * (HQ / 4));
    float acc[kR];
#pragma unroll
    for (int n = 0; n < kR; ++n) acc[n] = 0.f;
    // eight hidden units (two Philox blocks) at a time; a warp whose 32 rows
    // hold no running trial skips the work
    const bool warp_live = __any_sync(kFull, active);
#pragma unroll
    for (int c = 0; c < HQ / 8; ++c) {
      if (!warp_live) break;
      float e[8];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float4 z = normals4(noise_block_rk(p.rk, tg, 0u, blk0 + (uint32_t)(2 * c + b)));
        e[4 * b] = z.x;
        e[4 * b + 1] = z.y;
        e[4 * b + 2] = z.z;
        e[4 * b + 3] = z.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int h = q * HQ + 8 * c + i;
        float& sv = s[8 * c + i];
        const float y = lg_h(sv);
        sv = fmaf(keep, sv, fmaf(p.noise, e[i], p.rate * net_sm[h * kRows + r]));
#pragma unroll
        for (int n = 0; n < kR; ++n) acc[n] = fmaf(W[n * H + h], y, acc[n]);
      }
    }
#pragma unroll
    for (int n = 0; n < kR; ++n) part[(q * kR + n) * kRows + r] = acc[n];
    __syncthreads();

    // ---- response units 4q .. 4q+3 of every trial (all quarters)
    if (warp_live) {
      const float4 zr = normals4(noise_block_rk(
          p.rk, tg, 0u, (uint32_t)k * (uint32_t)(L::U / 4) + (uint32_t)(H / 4 + q)));
      const float e4[4] = {zr.x, zr.y, zr.z, zr.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = 4 * q + j;
        const float net = ((part[(0 * kR + n) * kRows + r] + part[(1 * kR + n) * kRows + r]) +
                           part[(2 * kR + n) * kRows + r]) + part[(3 * kR + n) * kRows + r];
        sr[j] = fmaf(keep, sr[j], fmaf(p.rate, net, p.noise * e4[j]));
        sh.yr[n][r] = lg_r(sr[j]);
      }
    }
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
}

template <int H>
cudaError_t launch_rows(const WideParams& p, cudaStream_t s) {
  using L = RowLay<H>;
  const size_t smem = L::WIN_OFF + (size_t)H * (p.S + p.T) * 4;
  cudaError_t e = smem_limit((const void*)wide_rows_kernel<H>, (int)smem);
  if (e != cudaSuccess) return e;
  long long grid = (p.n + kRows - 1) / kRows;
  const long long cap = (long long)num_sms();
  if (grid > cap) grid = cap;
  wide_rows_kernel<H><<<(unsigned)grid, kRowThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Time-blocked tensor-core form.
//
// The hidden layer takes no input from the response layer (the network is
// feed-forward and its inputs are clamped), so a trial's hidden trajectory
// does not depend on how its responses evolve. The CTA therefore advances
// kSlots trials by kBlkSteps steps at a time: the 128 rows of one MMA tile are
// (step j, slot s), row = kSlots j + s, and one tcgen05.mma chain gives every
// row's response net input at once.
//   1. hidden: thread (slot s, quad q) owns hidden units 4q .. 4q+3 of the
//      slot's trial (state and constant net input in registers) and runs them
//      through the block's kBlkSteps steps, writing y(t-1) of each step as a
//      bfloat16 hi + lo pair into A row (j, s);
//   2. lane 0 of each of the first kAcc warps issues one accumulation chain
//      of the MMAs D = A W^T (K = 2H, split in kAcc parts) into TMEM, while
//      the other warps draw the response units' noise of every row and the
//      next block's first-step normals;
//   3. response (warps 0-3, one thread per row, which is its TMEM lane):
//      u = rate D + noise eps per row, the response integrators advance
//      through the block's steps (thread (slot, unit pair)), and the stop rule
//      is applied at every step (thread (slot, step)); the first stopping
//      step of a slot ends its trial, and the slot takes the next trial.
// A slot's steps after its stopping step are computed and discarded (half a
// block per trial on average). Finished slots are refilled at every block
// boundary, so a CTA never runs idle rows for a whole launch and the grid
// spans every SM.
constexpr int kSlots = 16;
constexpr int kBlkSteps = 8;
static_assert(kSlots * kBlkSteps == kRows, "one MMA tile per block");
constexpr int kUYStep = kSlots * 20 + 4;   // floats per step in the u/y scratch (padded)
// independent MMA accumulation chains, each issued by lane 0 of its own warp
// (a thread takes a few hundred cycles to issue one of these MMAs): eight at
// H = 256, four below (where eight cost the response phase spills)
template <int H>
constexpr int acc_chains() { return H == 256 ? 8 : 4; }

template <int H>
struct BLay {
  static constexpr int Q = H / 4;                       // unit quads
  static constexpr int K2 = 2 * H;
  static constexpr int U = H + kR;
  static constexpr int THREADS = kSlots * Q > kRows ? kSlots * Q : kRows;
  static constexpr int ACC = acc_chains<H>();
  // offsets from the 1024-byte aligned start of dynamic shared memory
  static constexpr uint32_t B_OFF = 0;
  static constexpr uint32_t B_BYTES = kR * K2 * 2;      // bf16 W image, 16 x K2, swizzled
  static constexpr uint32_t A_OFF = (B_BYTES + 1023) / 1024 * 1024;
  static constexpr uint32_t A_BYTES = kRows * K2 * 2;   // bf16 128 x K2, swizzled
  static constexpr uint32_t UY_OFF = A_OFF + A_BYTES;   // [kBlkSteps][kSlots][20] floats
  static constexpr uint32_t UY_BYTES = kBlkSteps * kUYStep * 4;
  static constexpr uint32_t RN_OFF = UY_OFF + UY_BYTES;   // response noise [128][20] floats
  static constexpr uint32_t RN_BYTES = kRows * 20 * 4;
  static constexpr uint32_t BYTES = RN_OFF + RN_BYTES + 1024;   // + alignment slack
};

// K-major operand descriptor in the 128-byte swizzled layout: 8-row groups
// 1024 bytes apart (the leading byte offset is not used by this layout).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  d |= (uint64_t)2 << 61;   // 128-byte swizzle
  return d;
}

// Hidden net input of every condition: table[c][h] = sum_j W_in[h][j] c_j,
// accumulated in input order with fused multiply-adds.
__global__ void wide_net_table(const float* __restrict__ w_in, const float* __restrict__ cond,
                               int nin, int H, float* __restrict__ table) {
  const int c = blockIdx.x, h = threadIdx.x;
  if (h >= H) return;
  const float* w = w_in + (size_t)h * nin;
  const float* ci = cond + (size_t)c * nin;
  float acc = 0.f;
  for (int j = 0; j < nin; ++j) acc = fmaf(__ldg(w + j), __ldg(ci + j), acc);
  table[(size_t)c * H + h] = acc;
}

struct BlockShared {
  uint64_t bar_load;
  uint64_t bar_mma;
  uint32_t tmem_base;
  int fail;
  long long slot[kSlots];     // local trial index, or -1
  int kstep[kSlots];          // steps the slot's trial took before this block
  int fresh[kSlots];          // the trial starts with this block
  int finished[kSlots];
  long long r0, r1;           // unused hand-out indices r0 .. r0 + n0 - 1, then r1 .. r1 + n1 - 1
  int n0, n1;
  int any;                    // a slot holds a trial after the refill
};

__device__ __forceinline__ void bar_sync_named(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <int H>
__global__ void __launch_bounds__(BLay<H>::THREADS, 1) wide_block_kernel(WideParams p) {
  using L = BLay<H>;
  constexpr int Q = L::Q;
  constexpr int kAcc = L::ACC;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ BlockShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the swizzled operands need 1024-byte alignment
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* uy = reinterpret_cast<float*>(smem + L::UY_OFF);
  float* rnoise = reinterpret_cast<float*>(smem + L::RN_OFF);   // [128 rows][20]
  unsigned char* A = smem + L::A_OFF;

  // hidden role: (slot, quad), a warp holding 2 slots x 16 consecutive quads,
  // so that a warp whose two slots are empty skips the step work (at the end of
  // a launch); a half-warp's 8-byte stores cover one row's 16 swizzled chunks
  const int hs = 2 * (warp & 7) + (lane >> 4);
  const int hq = 16 * (warp >> 3) + (lane & 15);
  const bool hidden = hq < Q;

  if (warp == 0) {
    tmem_alloc(&sh.tmem_base, kAcc * kR < 32 ? 32 : kAcc * kR);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&sh.bar_load, 1);
    mbar_init(&sh.bar_mma, kAcc);
    fence_mbar_init();
    sh.fail = 0;
    sh.r0 = sh.r1 = 0;
    sh.n0 = sh.n1 = 0;
    mbar_expect_tx(&sh.bar_load, L::B_BYTES);
    bulk_g2s(smem + L::B_OFF, p.w_resp_bf16, L::B_BYTES, &sh.bar_load);
  }
  // first trials: one hand-out of kSlots indices
  if (warp == 0) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.cursor, (unsigned long long)kSlots);
    base = __shfl_sync(kFull, base, 0);
    if (lane < kSlots) {
      const long long f = (long long)base + lane;
      sh.slot[lane] = f < p.n ? f : -1;
      sh.kstep[lane] = 0;
      sh.fresh[lane] = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!mbar_wait(&sh.bar_load, 0)) {
    atomicExch(p.status, 1);
    sh.fail = 1;
  }
  const uint32_t tmem_d = sh.tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const float keep = 1.0f - p.rate;
  const Logistic lg_h = Logistic::of(p.gain_h, p.bias_h), lg_r = Logistic::of(p.gain_r, p.bias_r);

  float s[4] = {0.f, 0.f, 0.f, 0.f}, net[4] = {0.f, 0.f, 0.f, 0.f};   // hidden role (net: rate net)
  float4 zpre = make_float4(0.f, 0.f, 0.f, 0.f);
  bool pre_ok = false;
  float sr[2] = {0.f, 0.f};                                           // response role
  unsigned long long pf = 0;                                          // thread 0: prefetch
  bool prefetched = false;
  uint32_t phase = 0;
  __syncthreads();

  while (true) {
    // ---------------------------------------------------------------- 1.
    const long long ht = sh.slot[hs];
    const int hk = sh.kstep[hs];
    // rows (j, hs) of this thread's units: hi and lo halves, 2048 bytes per step
    unsigned char* a_hi = A + sw128_off(hs, 4 * hq, kRows);
    unsigned char* a_lo = A + sw128_off(hs, H + 4 * hq, kRows);
    if (hidden && ht >= 0) {
      const uint32_t tg = p.trial0 + (uint32_t)ht;
      if (sh.fresh[hs]) {
        const long long g = (long long)p.trial0 + ht;
        const float4 nt = __ldg(reinterpret_cast<const float4*>(
            p.net_table + (size_t)((g / p.cond_block) % p.n_cond) * H + 4 * hq));
        // rate net, constant through the trial (the hidden layer's inputs are
        // clamped), formed once
        net[0] = p.rate * nt.x;
        net[1] = p.rate * nt.y;
        net[2] = p.rate * nt.z;
        net[3] = p.rate * nt.w;
#pragma unroll
        for (int i = 0; i < 4; ++i) s[i] = 0.f;
      }
      // one step: y(t-1) of the thread's units into A row (j, hs), then the update
      // every step of the block is taken without a test against max_steps: a
      // running trial starts a block below it and stops at it at the latest,
      // and the rows after a trial's stopping step are never read
      auto step = [&](int j, float4 z) {
        float y[4];
        const float e[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          y[i] = lg_h(s[i]);
          s[i] = fmaf(keep, s[i], fmaf(p.noise, e[i], net[i]));
        }
        uint2 hi, lo;
        split2(y[0], y[1], hi.x, lo.x);
        split2(y[2], y[3], hi.y, lo.y);
        *reinterpret_cast<uint2*>(a_hi + 2048 * j) = hi;
        *reinterpret_cast<uint2*>(a_lo + 2048 * j) = lo;
      };
      uint32_t blk = (uint32_t)hk * (uint32_t)(L::U / 4) + (uint32_t)hq;
      // the first step's normals were drawn during the previous block's MMA
      // when the slot kept its trial
      if (!(pre_ok && !sh.fresh[hs])) zpre = normals4(noise_block_rk(p.rk, tg, 0u, blk));
      step(0, zpre);
#pragma unroll 2
      for (int j = 1; j < kBlkSteps; ++j) {
        blk += (uint32_t)(L::U / 4);
        step(j, normals4(noise_block_rk(p.rk, tg, 0u, blk)));
      }
    }
    // (an empty slot's rows keep earlier values: their products are not read)
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();

    // ---------------------------------------------------------------- 2.
    // K is split in kAcc parts, each an independent accumulation chain in its
    // own TMEM columns, issued by lane 0 of warp c and committed to the same
    // barrier; the response threads add the parts
    if (warp < kAcc && lane == 0 && !sh.fail) {
      tc_fence_after();
      // K slice kc = 16 kc .. 16 kc + 15: its 64-element atom, then 32 bytes per
      // slice inside the atom; the descriptors' address fields (bytes / 16)
      // advance by constants, so every MMA is issued from precomputed operands
      const uint64_t da = smem_desc_sw128(smem_u32(A)), db = smem_desc_sw128(smem_u32(smem + L::B_OFF));
      constexpr uint32_t idesc = mma_idesc(kRows, kR);
      constexpr int per = L::K2 / 16 / kAcc;
      const uint32_t dcol = tmem_d + (uint32_t)(warp * kR);
#pragma unroll
      for (int i = 0; i < per; ++i) {
        const int kc = warp * per + i;
        const uint64_t oa = (uint64_t)((kc >> 2) * (kRows * 128) + (kc & 3) * 32) >> 4;
        const uint64_t ob = (uint64_t)((kc >> 2) * (kR * 128) + (kc & 3) * 32) >> 4;
        mma_bf16(dcol, da + oa, db + ob, idesc, i > 0 ? 1u : 0u);
      }
      mma_commit(&sh.bar_mma);
    }

    // while the MMA runs: the normals of the next block's first step, for a
    // slot that keeps its trial (used only if it does), drawn by the warps
    // that issue no MMA (the issuing lanes' warps take no other work here:
    // a thread takes a few hundred cycles to issue each MMA)
    pre_ok = false;
    if (warp >= kAcc && hidden && ht >= 0 && hk + kBlkSteps < p.max_steps) {
      zpre = normals4(noise_block_rk(p.rk, p.trial0 + (uint32_t)ht, 0u,
                                     (uint32_t)(hk + kBlkSteps) * (uint32_t)(L::U / 4) +
                                         (uint32_t)hq));
      pre_ok = true;
    }
    // and the response units' noise of every row, sigma eps, by the threads
    // of the warps that issue no MMA: item (row, Philox block i) draws units
    // 4 i .. 4 i + 3 of the row's step
    constexpr int kNoise0 = 32 * kAcc < L::THREADS - kRows ? 32 * kAcc : L::THREADS - kRows;
    for (int w = tid - kNoise0; w >= 0 && w < 4 * kRows; w += L::THREADS - kNoise0) {
      const int row = w & (kRows - 1), i = w >> 7;
      const int rs = row & (kSlots - 1), rj = row / kSlots;
      const long long rt = sh.slot[rs];
      const int rst = sh.kstep[rs] + rj;
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rt >= 0 && rst < p.max_steps)
        z = normals4(noise_block_rk(p.rk, p.trial0 + (uint32_t)rt, 0u,
                                    (uint32_t)rst * (uint32_t)(L::U / 4) + (uint32_t)(H / 4 + i)));
      const float2 lo2 = __fmul2_rn(f2(p.noise), f2(z.x, z.y));
      const float2 hi2 = __fmul2_rn(f2(p.noise), f2(z.z, z.w));
      *reinterpret_cast<float4*>(rnoise + row * 20 + 4 * i) = make_float4(lo2.x, lo2.y, hi2.x, hi2.y);
    }
    __syncthreads();   // every row's response noise is in shared memory

    // ---------------------------------------------------------------- 3.
    if (tid < kRows) {
      // (a) row (step j, slot s): u = rate D + noise eps
      const int rs = tid & (kSlots - 1), rj = tid / kSlots;
      // prefetch a hand-out of kSlots indices while the MMA runs, whenever the
      // indices in hand could not refill every slot
      if (tid == 0 && sh.n1 == 0 && sh.n0 < kSlots) {
        pf = atomicAdd(p.cursor, (unsigned long long)kSlots);
        prefetched = true;
      }
      if (!sh.fail && !mbar_wait(&sh.bar_mma, phase)) {
        atomicExch(p.status, 1);
        sh.fail = 1;
      }
      __syncwarp();
      tc_fence_after();
      // the chains summed in order, ((c0 + c1) + c2) + c3, and u = rate D +
      // sigma eps, two columns at a time on the paired FP32 instructions
      float d[16];
      tmem_ld16(tmem_d + lane_base, d);
      // (16 columns per load at H = 256; 8 below, where the wider load
      // costs the hidden role's registers spills)
      constexpr int kLd = H == 256 ? 16 : 8;
#pragma unroll
      for (int c = 1; c < kAcc; ++c)
#pragma unroll
        for (int h = 0; h < 16 / kLd; ++h) {
          float d2[kLd];
          if constexpr (kLd == 16)
            tmem_ld16(tmem_d + lane_base + (uint32_t)(c * kR), d2);
          else
            tmem_ld8(tmem_d + lane_base + (uint32_t)(c * kR + 8 * h), d2);
#pragma unroll
          for (int n = 0; n < kLd; n += 2) {
            const float2 t = __fadd2_rn(f2(d[kLd * h + n], d[kLd * h + n + 1]), f2(d2[n], d2[n + 1]));
            d[kLd * h + n] = t.x;
            d[kLd * h + n + 1] = t.y;
          }
        }
      tc_fence_before();
      float* u = uy + rj * kUYStep + rs * 20;
      const float* ne = rnoise + tid * 20;
#pragma unroll
      for (int n = 0; n < kR; n += 4) {
        const float4 e = *reinterpret_cast<const float4*>(ne + n);
        const float2 a = __ffma2_rn(f2(p.rate), f2(d[n], d[n + 1]), f2(e.x, e.y));
        const float2 b = __ffma2_rn(f2(p.rate), f2(d[n + 2], d[n + 3]), f2(e.z, e.w));
        *reinterpret_cast<float4*>(u + n) = make_float4(a.x, a.y, b.x, b.y);
      }
      bar_sync_named(1, kRows);

      // (b) slot s2, units 2 p2, 2 p2 + 1: the integrators through the block's steps
      {
        const int s2 = tid >> 3, p2 = tid & 7;
        if (sh.fresh[s2]) {
          sr[0] = 0.f;
          sr[1] = 0.f;
        }
        if (sh.slot[s2] >= 0) {
          // both units on the paired FP32 instructions: the same roundings as
          // fmaf(keep, s, u) and the logistic's fma and add
          float2 sv = f2(sr[0], sr[1]);
#pragma unroll
          for (int j = 0; j < kBlkSteps; ++j) {
            float2* q2 = reinterpret_cast<float2*>(uy + j * kUYStep + s2 * 20 + 2 * p2);
            sv = __ffma2_rn(f2(keep), sv, *q2);
            const float2 t = __ffma2_rn(sv, f2(lg_r.c1), f2(lg_r.c0));
            float e0, e1, y0, y1;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(t.x));
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(t.y));
            const float2 den = __fadd2_rn(f2(1.0f), f2(e0, e1));
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(den.x));
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(den.y));
            *q2 = f2(y0, y1);
          }
          sr[0] = sv.x;
          sr[1] = sv.y;
        }
      }
      bar_sync_named(1, kRows);

      // (c) slot s3 at step j3: the stop rule; the first stopping step ends the trial
      {
        const int s3 = tid >> 3, j3 = tid & 7;
        const long long t3 = sh.slot[s3];
        const int k3 = sh.kstep[s3];
        const int st1 = k3 + j3 + 1;   // 1-based step
        const float* yv = uy + j3 * kUYStep + s3 * 20;
        int best = 0;
        float v1 = yv[0];
#pragma unroll
        for (int n = 1; n < kR; ++n) {
          const float v = yv[n];
          if (v > v1) {
            v1 = v;
            best = n;
          }
        }
        float v2 = -INFINITY;
#pragma unroll
        for (int n = 0; n < kR; ++n)
          if (n != best) v2 = fmaxf(v2, yv[n]);
        const bool hit = v1 - v2 > p.stop_threshold;
        const bool stop_here = t3 >= 0 && st1 <= p.max_steps && (hit || st1 >= p.max_steps);
        const unsigned m = __ballot_sync(kFull, stop_here);
        const unsigned grp = (m >> (lane & 24)) & 0xFFu;
        const bool first = stop_here && (grp & ((1u << j3) - 1u)) == 0u;
        if (first) {
          p.choice[t3] = hit ? (int8_t)best : (int8_t)-1;
          p.step[t3] = hit ? st1 : p.max_steps;
          if (p.yout)
#pragma unroll
            for (int n = 0; n < kR; ++n) p.yout[(size_t)t3 * kR + n] = yv[n];
        }
        if (j3 == 0) sh.finished[s3] = grp != 0u;
      }
      bar_sync_named(1, kRows);

      // (d) refill: finished slots take the next hand-out indices in slot order,
      // from the range in hand (r0) and then the prefetched one (r1)
      if (warp == 0) {
        const bool fin = lane < kSlots && sh.finished[lane];
        const unsigned fm = __ballot_sync(kFull, fin);
        const int rank = __popc(fm & ((1u << lane) - 1u));
        const int used = __popc(fm);
        long long r0 = sh.r0, r1 = sh.r1;
        int n0 = sh.n0, n1 = sh.n1;
        const int got = __shfl_sync(kFull, prefetched ? 1 : 0, 0);
        const unsigned long long pb = __shfl_sync(kFull, pf, 0);
        if (got) {
          r1 = (long long)pb;
          n1 = kSlots;
        }
        if (fin) {
          const long long f = rank < n0 ? r0 + rank : r1 + (rank - n0);
          sh.slot[lane] = f < p.n ? f : -1;
          sh.kstep[lane] = 0;
          sh.fresh[lane] = 1;
        } else if (lane < kSlots) {
          sh.kstep[lane] += kBlkSteps;
          sh.fresh[lane] = 0;
        }
        __syncwarp();
        const unsigned live = __ballot_sync(kFull, lane < kSlots && sh.slot[lane] >= 0);
        if (lane == 0) {
          sh.any = live != 0u;
          if (used <= n0) {
            sh.r0 = r0 + used;
            sh.n0 = n0 - used;
            sh.r1 = r1;
            sh.n1 = n1;
          } else {
            sh.r0 = r1 + (used - n0);
            sh.n0 = n1 - (used - n0);
            sh.r1 = 0;
            sh.n1 = 0;
          }
        }
        prefetched = false;
      }
    }
    phase ^= 1u;
    __syncthreads();
    if (!sh.any || sh.fail) break;
  }

  // ---- tear-down
  __syncthreads();
  if (sh.fail) {
    if (tid == 0) mbar_wait(&sh.bar_mma, phase ^ 1u);
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(sh.tmem_base, kAcc * kR < 32 ? 32 : kAcc * kR);
}

template <int H>
cudaError_t launch_block(const WideParams& p, cudaStream_t s) {
  using L = BLay<H>;
  const size_t smem = L::BYTES;
  cudaError_t e = smem_limit((const void*)wide_block_kernel<H>, (int)smem);
  if (e != cudaSuccess) return e;
  wide_net_table<<<(unsigned)p.n_cond, H, 0, s>>>(p.w_in, p.cond, p.S + p.T, H, p.net_table);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  long long grid = (p.n + kSlots - 1) / kSlots;
  const long long cap = (long long)num_sms();   // one CTA per SM (its shared memory)
  if (grid > cap) grid = cap;
  wide_block_kernel<H><<<(unsigned)grid, L::THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t wide_smem_bytes(int H, int nin, bool tc) {
  if (tc) {   // time-blocked form: W image, A tile, u/y scratch, alignment slack
    (void)nin;
    const size_t a_off = ((size_t)kR * 2 * H * 2 + 1023) / 1024 * 1024;
    return a_off + (size_t)kRows * 2 * H * 2 + (size_t)kBlkSteps * kUYStep * 4 +
           (size_t)kRows * 20 * 4 + 1024;
  }
  const size_t part_off = ((size_t)kR * H * 4 + 1023) / 1024 * 1024;
  return part_off + (size_t)(4 * kR * kRows + H * kRows) * 4 + (size_t)H * nin * 4;
}

void wide_b_image(const uint16_t* w_bf16, int H, uint16_t* img) {
  // B operand image: row n of K2 = 2H elements is [W[n][0..H) | W[n][0..H)]
  // (the hi and lo halves of the activations meet the same weights), in the
  // 128-byte swizzled K-major layout of the tensor-core tile
  const int K2 = 2 * H;
  for (int n = 0; n < kR; ++n)
    for (int k = 0; k < K2; ++k) img[sw128_off(n, k, kR) / 2] = w_bf16[(size_t)n * H + (k % H)];
}

cudaError_t launch_wide(const WideParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  (void)cfg;
  if (p.n <= 0) return cudaSuccess;
  const bool tc = mode == 0;
  switch (p.H) {
    case 64: return tc ? launch_block<64>(p, s) : launch_rows<64>(p, s);
    case 128: return tc ? launch_block<128>(p, s) : launch_rows<128>(p, s);
    case 192: return tc ? launch_block<192>(p, s) : launch_rows<192>(p, s);
    case 256: return tc ? launch_block<256>(p, s) : launch_rows<256>(p, s);
  }
  return cudaErrorNotSupported;
}

}  // namespace dg
