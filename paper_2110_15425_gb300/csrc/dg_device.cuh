// Device building blocks shared by every kernel of the library: counter-based
// random numbers and warp-level trial scheduling.
//
// Random draws (Sec. 3.6 asks that every evaluation draw reproducible,
// independent numbers; the paper restores a per-evaluation PRNG state on each
// call, which costs ~7.5 kB per GPU thread). Here the generator is
// Philox4x32-10 (Salmon et al., SC'11) with no state at all: block b of the
// stream of (seed, trial, candidate) is Philox(counter = (trial, candidate,
// b, 0), key = (seed lo, seed hi)). Normal d of the stream is lane d & 3 of
// the Box-Muller transform of block d >> 2.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dg {

constexpr unsigned kFull = 0xffffffffu;

// One Philox4x32-10 block. Each round multiplies words 0 and 2 by the two
// round multipliers, then mixes the high halves with words 1 and 3 and the
// key; the key advances by the two Weyl increments between rounds.
__host__ __device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit multiply gives both halves of each product
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same block with the round keys precomputed (dg::PhiloxKeys).
template <typename Keys>
__device__ __forceinline__ uint4 philox_rk(uint4 c, const Keys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk.k[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

// Round keys formed where they are used from the key pair (one add each),
// for code that holds a different key in each lane and has no registers to
// spare for the twenty round keys; same keys, same blocks as dg::PhiloxKeys.
struct KeyPair {
  struct Rounds {
    uint32_t k0, k1;
    __device__ __forceinline__ uint32_t operator[](int i) const {
      return (i & 1) ? k1 + (uint32_t)(i >> 1) * 0xBB67AE85u : k0 + (uint32_t)(i >> 1) * 0x9E3779B9u;
    }
  } k;
};

template <typename Keys>
__device__ __forceinline__ uint4 noise_block_rk(const Keys& rk, uint32_t trial, uint32_t cand,
                                                uint32_t block) {
  return philox_rk(make_uint4(trial, cand, block, 0u), rk);
}

__device__ __forceinline__ uint4 noise_block(uint32_t k0, uint32_t k1, uint32_t trial,
                                             uint32_t cand, uint32_t block) {
  return philox(make_uint4(trial, cand, block, 0u), k0, k1);
}

// u = ((w >> 9) + 1/2) 2^-23: the 24-bit odd numerator is exact in binary32,
// so the fma below is exact.
__device__ __forceinline__ float u01(uint32_t w) {
  return fmaf(__uint2float_rn(w >> 9), 0x1p-23f, 0x1p-24f);
}

// The 23 payload bits of w as the binary32 value 1 + (w >> 9) 2^-23 in [1, 2);
// u = that - (1 - 2^-24) equals ((w >> 9) + 1/2) 2^-23 exactly.
__device__ __forceinline__ float one_plus(uint32_t w) { return __uint_as_float((w >> 9) | 0x3F800000u); }

// The hardware approximations (MUFU) in their flush-to-zero forms. Every
// argument and result below is a normal binary32 number or zero (u >= 2^-24,
// -2 ln u >= 2^-23, angles of magnitude >= 2 pi 2^-24), where the two forms
// return the same bits; the flush-to-zero form saves the subnormal
// range fix-up instructions around each approximation.
__device__ __forceinline__ float approx_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_sin(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float approx_cos(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// -2 ln(u) for u in (0, 1). The hardware log2 approximation has a small
// absolute error, which is a large relative error when u is close to 1 and
// ln(u) is tiny; there the Taylor series -2 ln(1 - v) = 2 (v + v^2/2 + v^3/3
// + ...) in v = 1 - u (exact in binary32 for u >= 1/2) is used instead: for
// v < 2^-6 five terms leave a relative truncation error below 2e-10.
__device__ __forceinline__ float neg2_log_u01(float u) {
  const float v = 1.0f - u;
  float r = -1.38629436111989062f * approx_lg2(u);   // -2 ln 2
  if (v < 0x1p-6f)  // taken for 1 draw in 64
    r = v * fmaf(v, fmaf(v, fmaf(v, fmaf(v, 0.4f, 0.5f), 2.0f / 3.0f), 1.0f), 2.0f);
  return r;
}

// Box-Muller (1958): radius sqrt(-2 ln u_a) from the first word, angle
// 2 pi u_b from the second. The angle is taken as 2 pi (u_b - 1/2) in
// (-pi, pi) (u_b - 1/2 is exact), which flips the sign of both sine and
// cosine, so the hardware sine/cosine see a reduced argument.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float y = neg2_log_u01(one_plus(wa) - 0.99999994039535522f);   // 1 - 2^-24
  const float r = y * approx_rsqrt(y);
  // u_b - 1/2 = (one_plus(w_b) - 3/2) + 2^-24, both steps exact; the fma
  // rounds 2 pi (u_b - 1/2) once, as a plain product of the exact difference
  // would (2 pi 2^-24 is exact)
  const float ang =
      fmaf(6.28318530717958648f, one_plus(wb) - 1.5f, 6.28318530717958648f * 0x1p-24f);
  z0 = -r * approx_cos(ang);
  z1 = -r * approx_sin(ang);
}

// Two Box-Muller pairs (words x, y and z, w) evaluated side by side: every
// FP32 add, multiply and fma of box_muller above done once for both pairs by
// the paired instructions of this architecture, which round each component
// exactly as the scalar instruction does, so the normals keep their bits.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float4 normals4(uint4 w) {
  const float2 u = __fadd2_rn(f2(one_plus(w.x), one_plus(w.z)), f2(-0.99999994039535522f));
  const float2 v = __fadd2_rn(f2(1.0f), f2(-u.x, -u.y));
  // -2 ln u from the hardware log2, or the series in v = 1 - u near u = 1
  const float2 y0 = __fmul2_rn(f2(-1.38629436111989062f), f2(approx_lg2(u.x), approx_lg2(u.y)));
  float2 q = __ffma2_rn(v, f2(0.4f), f2(0.5f));
  q = __ffma2_rn(v, q, f2(2.0f / 3.0f));
  q = __ffma2_rn(v, q, f2(1.0f));
  q = __ffma2_rn(v, q, f2(2.0f));
  q = __fmul2_rn(v, q);
  const float2 y = f2(v.x < 0x1p-6f ? q.x : y0.x, v.y < 0x1p-6f ? q.y : y0.y);
  const float2 r = __fmul2_rn(y, f2(approx_rsqrt(y.x), approx_rsqrt(y.y)));
  const float2 ang = __ffma2_rn(f2(6.28318530717958648f),
                                __fadd2_rn(f2(one_plus(w.y), one_plus(w.w)), f2(-1.5f)),
                                f2(6.28318530717958648f * 0x1p-24f));
  const float2 nr = f2(-r.x, -r.y);
  const float2 zc = __fmul2_rn(nr, f2(approx_cos(ang.x), approx_cos(ang.y)));
  const float2 zs = __fmul2_rn(nr, f2(approx_sin(ang.x), approx_sin(ang.y)));
  return make_float4(zc.x, zs.x, zc.y, zs.y);
}

__device__ __forceinline__ float pick4(const float4& z, uint32_t lane) {
  const float a = (lane & 1u) ? z.y : z.x;
  const float b = (lane & 1u) ? z.w : z.z;
  return (lane & 2u) ? b : a;
}

// Drift-diffusion state in 64-bit fixed point with 40 fractional bits: FP32
// sums inside each 4-step Philox block are rounded once to fixed point and
// added exactly, so the state does not depend on the order of those additions.
// The conversions run on the double-precision unit of this GPU; exact
// single-precision constructions of the same roundings were measured slower.
constexpr float kFixScale = 1099511627776.0f;       // 2^40
constexpr float kFixInv = 9.094947017729282e-13f;   // 2^-40

__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * kFixScale); }

__device__ __forceinline__ float from_fix(long long v) { return __ll2float_rn(v) * kFixInv; }

// Warp-aggregated fetch of trial ids from a global cursor: every lane of the
// warp must call it; lanes with `need` get consecutive new ids (or -1 when no
// lane needs one). One atomic per warp per call.
__device__ __forceinline__ long long fetch_trial(unsigned long long* cursor, bool need) {
  const unsigned mask = __ballot_sync(kFull, need);
  if (mask == 0u) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  if (!need) return -1;
  return (long long)(base + (unsigned long long)__popc(mask & ((1u << lane) - 1u)));
}

// Multi-job launches: copy the job table from the kernel parameter into
// shared memory (one barrier), and find the job holding entry f of the
// concatenated trial list (the last job whose start is at most f; starts
// ascend from 0).
__device__ __forceinline__ void copy_jobs(const MultiJobTable& tab, MultiJob* s_job) {
  static_assert(sizeof(MultiJob) % 8 == 0, "job records copy as 8-byte words");
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(tab.jobs);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(s_job);
  const int words = tab.n_jobs * (int)(sizeof(MultiJob) / 8);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// The job-table parameter of a kernel that runs one job or several.
template <bool MULTI>
struct TableOf {
  using type = MultiJobTable;
};
template <>
struct TableOf<false> {   // a single job carries no table
  struct type {};
};

__device__ __forceinline__ int multi_job_of(const MultiJob* s_job, int n_jobs, long long f) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_job[mid].start <= f) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// y = 1 / (1 + exp(-gain (s + bias))) = 1 / (1 + 2^(c1 s + c0)) with
// c1 = -gain log2(e), c0 = -gain bias log2(e): one fma, the hardware 2^x and
// reciprocal approximations (flush-to-zero forms: a subnormal 2^x adds
// nothing to 1, and a reciprocal of 1 + 2^x above 2^126 is 0 either way).
struct Logistic {
  float c1, c0;
  __device__ __forceinline__ static Logistic of(float gain, float bias) {
    const float l2e = 1.44269504088896341f;
    return Logistic{-gain * l2e, -(gain * bias) * l2e};
  }
  __device__ __forceinline__ float operator()(float s) const {
    float e, y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fmaf(s, c1, c0)));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(1.0f + e));
    return y;
  }
};

}  // namespace dg
