// Small layered logistic networks (the Botvinick Stroop model of Sec. 5), one
// thread per trial. Every logistic unit integrates with time averaging,
//   s <- (1 - rate) s + rate net + noise eps,  y = 1 / (1 + exp(-gain (s + bias))),
// and all units read the previous iteration's outputs (the current/previous
// output structures of Sec. 3.3), so the update is synchronous. Input layers
// are clamped, so their contribution to every net input is computed once per
// trial. A trial ends at the first step where the stop layer's largest output
// exceeds the second largest by more than the threshold.
//
// The per-thread unit state lives in shared memory laid out [unit][thread],
// so the dynamic unit indexing of an arbitrary small graph costs no local
// memory and no bank conflicts; the static layout (edges, gains, biases) is
// staged into shared memory once per block and read as broadcasts.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

struct NetSmem {
  float* y;      // [U][B] outputs of the previous step
  float* yn;     // [U][B] outputs of this step
  float* s;      // [U][B] integrator state
  float* net;    // [U][B] net input of this step
  float* netc;   // [U][B] constant (input-layer) part of the net input
};

__device__ __forceinline__ void net_begin(const NetParams& p, const NetLayout& L, long long t,
                                          NetSmem& m, int tid, int B) {
  const long long g = (long long)p.trial0 + t;  // global trial id
  const int cond = (int)((g / p.cond_block) % p.n_cond);
  const float* cin = p.cond + (size_t)cond * L.n_in;
  for (int u = 0; u < L.U; ++u) {
    float acc = 0.f;
    const float* w = p.w_in + (size_t)u * L.n_in;
    for (int q = 0; q < L.n_in; ++q) acc = fmaf(__ldg(w + q), __ldg(cin + q), acc);
    m.netc[u * B + tid] = acc;
    m.s[u * B + tid] = 0.f;
    m.y[u * B + tid] = logistic(L.gain[u], L.bias[u], 0.f);
  }
}

// One synchronous step k (0-based). Returns true when the stop rule fires.
__device__ __forceinline__ bool net_step(const NetParams& p, const NetLayout& L, uint32_t trial,
                                         int k, NetSmem& m, int tid, int B, int8_t& choice) {
  for (int u = 0; u < L.U; ++u) m.net[u * B + tid] = m.netc[u * B + tid];
  for (int e = 0; e < L.n_edges; ++e) {
    const int d = L.edge_dst[e], sidx = L.edge_src[e];
    m.net[d * B + tid] = fmaf(L.edge_w[e], m.y[sidx * B + tid], m.net[d * B + tid]);
  }
  const uint32_t d0 = (uint32_t)k * (uint32_t)L.U;
  float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int u = 0; u < L.U; ++u) {
    const uint32_t d = d0 + (uint32_t)u;
    if (u == 0 || (d & 3u) == 0u) z = normals4(noise_block(p.k0, p.k1, trial, 0u, d >> 2));
    const float e = pick4(z, d & 3u);
    const float sv = fmaf(1.0f - L.rate, m.s[u * B + tid],
                          fmaf(L.rate, m.net[u * B + tid], L.noise * e));
    m.s[u * B + tid] = sv;
    m.yn[u * B + tid] = logistic(L.gain[u], L.bias[u], sv);
  }
  float* tmp = m.y;
  m.y = m.yn;
  m.yn = tmp;
  // stop rule on the fresh outputs
  const float* ys = m.y + L.stop_off * B + tid;
  int best = 0;
  float v1 = ys[0];
  for (int i = 1; i < L.stop_size; ++i) {
    const float v = ys[i * B];
    if (v > v1) {
      v1 = v;
      best = i;
    }
  }
  float v2 = -INFINITY;
  for (int i = 0; i < L.stop_size; ++i)
    if (i != best) v2 = fmaxf(v2, ys[i * B]);
  if (v1 - v2 > L.stop_threshold) {
    choice = (int8_t)best;
    return true;
  }
  return false;
}

__device__ __forceinline__ void net_write(const NetParams& p, const NetLayout& L, long long t,
                                          int8_t c, int st, const NetSmem& m, int tid, int B) {
  p.choice[t] = c;
  p.step[t] = st;
  if (p.yout)
    for (int i = 0; i < L.stop_size; ++i)
      p.yout[(size_t)t * L.stop_size + i] = m.y[(L.stop_off + i) * B + tid];
}

// cursor == null: one thread per trial; otherwise a persistent grid that
// refills finished lanes from the cursor.
__global__ void __launch_bounds__(128) net_kernel(NetParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  NetLayout& L = *reinterpret_cast<NetLayout*>(smem);
  {
    const int words = (int)(sizeof(NetLayout) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(p.layout);
    uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int B = blockDim.x, tid = threadIdx.x;
  float* base = reinterpret_cast<float*>(smem + ((sizeof(NetLayout) + 15) / 16) * 16);
  const int U = p.U;
  NetSmem m{base, base + U * B, base + 2 * U * B, base + 3 * U * B, base + 4 * U * B};

  const bool persistent = p.cursor != nullptr;
  long long t;
  if (persistent) {
    t = fetch_trial(p.cursor, true);
  } else {
    t = (long long)blockIdx.x * B + tid;
  }
  bool active = t >= 0 && t < p.n;
  if (!persistent && !active) return;
  int k = 0;
  if (active) net_begin(p, L, t, m, tid, B);
  while (persistent ? __any_sync(kFull, active) : active) {
    bool finished = false;
    if (active) {
      int8_t c = -1;
      const bool hit = net_step(p, L, p.trial0 + (uint32_t)t, k, m, tid, B, c);
      ++k;
      if (hit || k >= L.max_steps) {
        net_write(p, L, t, hit ? c : (int8_t)-1, hit ? k : L.max_steps, m, tid, B);
        finished = true;
      }
    }
    if (persistent) {
      const long long nt = fetch_trial(p.cursor, finished);
      if (finished) {
        t = nt;
        active = t < p.n;
        k = 0;
        if (active) net_begin(p, L, t, m, tid, B);
      }
    } else if (finished) {
      active = false;
    }
  }
}

size_t net_smem_bytes(int U, int B) {
  return ((sizeof(NetLayout) + 15) / 16) * 16 + (size_t)5 * U * B * sizeof(float);
}

}  // namespace

cudaError_t launch_net(const NetParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  const int B = 128;
  const size_t smem = net_smem_bytes(p.U, B);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(net_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  NetParams q = p;
  long long grid;
  if (mode == 1 || p.cursor == nullptr) {
    q.cursor = nullptr;
    grid = (p.n + B - 1) / B;
  } else {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, net_kernel, B, smem);
    if (nb < 1) nb = 1;
    grid = cfg.grid > 0 ? cfg.grid : (long long)num_sms() * nb;
    const long long need = (p.n + B - 1) / B;
    if (grid > need) grid = need;
  }
  net_kernel<<<(unsigned)grid, B, smem, s>>>(q);
  return cudaGetLastError();
}

}  // namespace dg
