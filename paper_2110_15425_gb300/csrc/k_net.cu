// Small layered logistic networks (the Botvinick Stroop model of Sec. 5).
// Every logistic unit integrates with time averaging,
//   s <- (1 - rate) s + rate net + noise eps,  y = 1 / (1 + exp(-gain (s + bias))),
// and all units read the previous iteration's outputs (the current/previous
// output structures of Sec. 3.3), so the update is synchronous. Input layers
// are clamped, so their contribution to every net input is computed once per
// trial. A trial ends at the first step where the stop layer's largest output
// exceeds the second largest by more than the threshold.
//
// Net input of unit u: netc_u + sum_{d < D} w[u][d] y[src[u][d]], summed in d
// order (a dense table of incoming edges, padded with zero weights), so both
// forms below add the same terms in the same order and agree bit for bit.
//
// Batched form (net_group): a trial is a group of G lanes (G = next power of
// two >= units), lane u holding unit u; sender outputs arrive by shuffles,
// every lane draws its own unit's normal, and the stop test is a group
// reduction. A step costs one Philox block's latency instead of U sequential
// unit updates; groups refill from the trial cursor.
// Plain form (net_plain): one thread per trial with the unit state in shared
// memory laid out [unit][thread].
#include <cfloat>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

__device__ __forceinline__ float unit_noise(const NetParams& p, uint32_t trial, int k, int U,
                                            int u) {
  const uint32_t d = (uint32_t)k * (uint32_t)U + (uint32_t)u;
  return pick4(normals4(noise_block(p.k0, p.k1, trial, 0u, d >> 2)), d & 3u);
}

__device__ __forceinline__ float const_net(const NetParams& p, const NetLayout& L, long long t,
                                           int u) {
  const long long g = (long long)p.trial0 + t;  // global trial id
  const int cond = (int)((g / p.cond_block) % p.n_cond);
  const float* cin = p.cond + (size_t)cond * L.n_in;
  const float* w = p.w_in + (size_t)u * L.n_in;
  float acc = 0.f;
  for (int q = 0; q < L.n_in; ++q) acc = fmaf(__ldg(w + q), __ldg(cin + q), acc);
  return acc;
}

__device__ __forceinline__ void stage_layout(const NetParams& p, unsigned char* smem) {
  const int words = (int)(sizeof(NetLayout) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(p.layout);
  uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// ------------------------------------------------------------- batched ---

template <int G>
__global__ void __launch_bounds__(256) net_group(NetParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_layout(p, smem);
  const NetLayout& L = *reinterpret_cast<const NetLayout*>(smem);
  const int lane = threadIdx.x & 31;
  const int u = lane % G;                 // unit of this lane
  const int root = lane - u;
  const unsigned gmask = (G == 32 ? kFull : ((1u << G) - 1u)) << root;
  const bool real = u < L.U;
  const bool in_stop = u >= L.stop_off && u < L.stop_off + L.stop_size;
  const Logistic lg = Logistic::of(real ? L.gain[u] : 1.f, real ? L.bias[u] : 0.f);

  long long f = fetch_trial(p.cursor, u == 0);
  f = __shfl_sync(kFull, f, root);
  bool active = f >= 0 && f < p.n;
  long long t = f;
  int k = 0;
  float s = 0.f, y = lg(0.f), netc = 0.f;
  if (active && real) netc = const_net(p, L, t, u);
  while (__any_sync(kFull, active)) {
    bool finished = false;
    if (active) {
      // synchronous: every lane reads the step k outputs before any update
      float net = netc;
      for (int d = 0; d < L.D; ++d) {
        const int si = real ? L.src[u][d] : 0;
        const float yv = __shfl_sync(gmask, y, root + si);
        if (real) net = fmaf(L.w[u][d], yv, net);
      }
      if (real) {
        const float e = unit_noise(p, p.trial0 + (uint32_t)t, k, L.U, u);
        s = fmaf(1.0f - L.rate, s, fmaf(L.rate, net, L.noise * e));
        y = lg(s);
      }
      // top-1 (lowest index on ties) and top-2 of the stop layer
      float v1 = in_stop ? y : -FLT_MAX, v2 = -FLT_MAX;
      int i1 = in_stop ? u - L.stop_off : 1 << 20;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const float ov1 = __shfl_xor_sync(gmask, v1, o);
        const float ov2 = __shfl_xor_sync(gmask, v2, o);
        const int oi1 = __shfl_xor_sync(gmask, i1, o);
        if (ov1 > v1 || (ov1 == v1 && oi1 < i1)) {
          v2 = fmaxf(v1, ov2);
          v1 = ov1;
          i1 = oi1;
        } else {
          v2 = fmaxf(v2, ov1);
        }
      }
      ++k;
      const bool hit = v1 - v2 > L.stop_threshold;
      if (hit || k >= L.max_steps) {
        if (u == 0) {
          p.choice[t] = hit ? (int8_t)i1 : (int8_t)-1;
          p.step[t] = hit ? k : L.max_steps;
        }
        if (p.yout && in_stop) p.yout[(size_t)t * L.stop_size + (u - L.stop_off)] = y;
        finished = true;
      }
    }
    f = fetch_trial(p.cursor, finished && u == 0);
    f = __shfl_sync(kFull, f, root);
    if (finished) {
      active = f < p.n;
      t = f;
      k = 0;
      s = 0.f;
      y = lg(0.f);
      netc = (active && real) ? const_net(p, L, t, u) : 0.f;
    }
  }
}

// --------------------------------------------------------------- plain ---

__global__ void __launch_bounds__(128) net_plain(NetParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_layout(p, smem);
  const NetLayout& L = *reinterpret_cast<const NetLayout*>(smem);
  const int B = blockDim.x, tid = threadIdx.x;
  float* base = reinterpret_cast<float*>(smem + ((sizeof(NetLayout) + 15) / 16) * 16);
  const int U = L.U;
  float* y = base;                 // [U][B]
  float* yn = base + U * B;
  float* s = base + 2 * U * B;
  float* netc = base + 3 * U * B;
  const long long t = (long long)blockIdx.x * B + tid;
  if (t >= p.n) return;
  for (int u = 0; u < U; ++u) {
    netc[u * B + tid] = const_net(p, L, t, u);
    s[u * B + tid] = 0.f;
    y[u * B + tid] = Logistic::of(L.gain[u], L.bias[u])(0.f);
  }
  const uint32_t trial = p.trial0 + (uint32_t)t;
  for (int k = 0; k < L.max_steps; ++k) {
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int u = 0; u < U; ++u) {
      float net = netc[u * B + tid];
      for (int d = 0; d < L.D; ++d) net = fmaf(L.w[u][d], y[L.src[u][d] * B + tid], net);
      // the same normal as unit_noise, reusing a block across consecutive units
      const uint32_t dn = (uint32_t)k * (uint32_t)U + (uint32_t)u;
      if (u == 0 || (dn & 3u) == 0u) z = normals4(noise_block(p.k0, p.k1, trial, 0u, dn >> 2));
      const float e = pick4(z, dn & 3u);
      const float sv = fmaf(1.0f - L.rate, s[u * B + tid], fmaf(L.rate, net, L.noise * e));
      s[u * B + tid] = sv;
      yn[u * B + tid] = Logistic::of(L.gain[u], L.bias[u])(sv);
    }
    float* tmp = y;
    y = yn;
    yn = tmp;
    const float* ys = y + L.stop_off * B + tid;
    int best = 0;
    float v1 = ys[0];
    for (int i = 1; i < L.stop_size; ++i)
      if (ys[i * B] > v1) {
        v1 = ys[i * B];
        best = i;
      }
    float v2 = -FLT_MAX;
    for (int i = 0; i < L.stop_size; ++i)
      if (i != best) v2 = fmaxf(v2, ys[i * B]);
    const bool hit = v1 - v2 > L.stop_threshold;
    if (hit || k + 1 >= L.max_steps) {
      p.choice[t] = hit ? (int8_t)best : (int8_t)-1;
      p.step[t] = hit ? k + 1 : L.max_steps;
      if (p.yout)
        for (int i = 0; i < L.stop_size; ++i) p.yout[(size_t)t * L.stop_size + i] = ys[i * B];
      return;
    }
  }
}

size_t layout_smem() { return ((sizeof(NetLayout) + 15) / 16) * 16; }

template <int G>
cudaError_t launch_group(const NetParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  const size_t smem = layout_smem();
  cudaError_t e =
      cudaFuncSetAttribute(net_group<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, net_group<G>, 256, smem);
  if (nb < 1) nb = 1;
  long long grid = cfg.grid > 0 ? cfg.grid : (long long)num_sms() * nb;
  const long long need = (p.n * G + 255) / 256;
  if (grid > need) grid = need;
  net_group<G><<<(unsigned)grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_net(const NetParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  if (mode == 1 || p.cursor == nullptr) {
    const int B = 128;
    const size_t smem = layout_smem() + (size_t)4 * p.U * B * sizeof(float);
    cudaError_t e =
        cudaFuncSetAttribute(net_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    net_plain<<<(unsigned)((p.n + B - 1) / B), B, smem, s>>>(p);
    return cudaGetLastError();
  }
  if (p.U <= 2) return launch_group<2>(p, cfg, s);
  if (p.U <= 4) return launch_group<4>(p, cfg, s);
  if (p.U <= 8) return launch_group<8>(p, cfg, s);
  if (p.U <= 16) return launch_group<16>(p, cfg, s);
  return launch_group<32>(p, cfg, s);
}

}  // namespace dg
