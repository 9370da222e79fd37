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
//
// Extended Stroop (Sec. 5): DDM nodes on the stop layer. When the network
// stops, node q takes drift_q = bias_q + sum_i w_qi y_i from the stop layer's
// outputs and integrates x += drift dt + sigma sqrt(dt) eps from 0 to |x| >= z_q
// (noise stream (trial, cand 1 + q); FP32 sums within each 4-step Philox block,
// 64-bit fixed point across blocks, as the DDM kernel). The trial's response
// is the first node to reach a bound (fewest steps, lower q on equal steps):
// choice 2 q + (upper bound), step = network steps + node steps; none: -1 and
// network steps + max_q node max. In the batched form lane q of the trial's
// group runs node q, one Philox block per loop iteration.
#include <cfloat>

#include "dg_device.cuh"
#include "dg_internal.h"
#include "dg_net.cuh"

namespace dg {

namespace {

// Normal k U + u of the trial's stream: only the Box-Muller pair that holds it.
__device__ __forceinline__ float unit_noise(const NetParams& p, uint32_t trial, int k, int U,
                                            int u) {
  const uint32_t d = (uint32_t)k * (uint32_t)U + (uint32_t)u;
  const uint4 w = noise_block_rk(p.rk, trial, 0u, d >> 2);
  const bool second = (d & 2u) != 0u;
  float z0, z1;
  box_muller(second ? w.z : w.x, second ? w.w : w.y, z0, z1);
  return (d & 1u) ? z1 : z0;
}

__device__ __forceinline__ void stage_layout(const NetParams& p, unsigned char* smem) {
  const int words = (int)(sizeof(NetLayout) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(p.layout);
  uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

__device__ __forceinline__ DdmNode ddm_node_begin(const NetLayout& L, int q, float drift) {
  return DdmNode{drift * L.ddm_dt[q], L.ddm_diffusion[q], L.ddm_z[q], L.ddm_max[q], 0ll, 0};
}

// Four steps of node q (one Philox block); true when the node has ended.
__device__ __forceinline__ bool ddm_node_block(const NetParams& p, uint32_t trial, int q,
                                               DdmNode& d, int& choice, int& step, float& x) {
  const float4 e = normals4(noise_block_rk(p.rk, trial, 1u + (uint32_t)q, (uint32_t)d.b));
  float pre[4];
  pre[0] = fmaf(d.diff, e.x, d.adt);
  pre[1] = pre[0] + fmaf(d.diff, e.y, d.adt);
  pre[2] = pre[1] + fmaf(d.diff, e.z, d.adt);
  pre[3] = pre[2] + fmaf(d.diff, e.w, d.adt);
  const float xb = from_fix(d.X);
  const int k = 4 * d.b;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float v = xb + pre[j];
    if (fabsf(v) >= d.z) {
      choice = v > 0.0f ? 1 : 0;
      step = k + j + 1;
      x = v;
      return true;
    }
    if (k + j + 1 == d.max) {
      choice = -1;
      step = d.max;
      x = v;
      return true;
    }
  }
  d.X += to_fix(pre[3]);
  ++d.b;
  return false;
}

// The trial's response from the nodes' (choice, step).
__device__ __forceinline__ void ddm_response(const NetLayout& L, const int* c, const int* st,
                                             int net_step, int8_t& choice, int32_t& step) {
  int first = -1;
  for (int q = 0; q < L.n_ddm; ++q)
    if (c[q] >= 0 && (first < 0 || st[q] < st[first])) first = q;
  if (first >= 0) {
    choice = (int8_t)(2 * first + c[first]);
    step = net_step + st[first];
  } else {
    int mx = 0;
    for (int q = 0; q < L.n_ddm; ++q) mx = max(mx, L.ddm_max[q]);
    choice = -1;
    step = net_step + mx;
  }
}

// ------------------------------------------------------------- batched ---

template <int G, bool EXT>
__global__ void __launch_bounds__(256) net_group(NetParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  stage_layout(p, smem);
  const NetLayout& L = *reinterpret_cast<const NetLayout*>(smem);
  const int lane = threadIdx.x & 31;
  const int u = lane % G;                 // unit of this lane (and DDM node, phase 1)
  const int root = lane - u;
  const unsigned gmask = (G == 32 ? kFull : ((1u << G) - 1u)) << root;
  const bool real = u < L.U;
  const bool in_stop = u >= L.stop_off && u < L.stop_off + L.stop_size;
  const Logistic lg = Logistic::of(real ? L.gain[u] : 1.f, real ? L.bias[u] : 0.f);
  // this lane's layout in registers: constants and up to kEdgeRegs incoming
  // edges (the rest, if any, are read from shared memory each step)
  constexpr int kEdgeRegs = 8;
  const int D = L.D;
  const float rate = L.rate, keep = 1.0f - L.rate, noise = L.noise, thr = L.stop_threshold;
  const int max_steps = L.max_steps, stop_off = L.stop_off;
  int esrc[kEdgeRegs];
  float ew[kEdgeRegs];
#pragma unroll
  for (int d = 0; d < kEdgeRegs; ++d) {
    esrc[d] = real && d < D ? L.src[u][d] : 0;
    ew[d] = real && d < D ? L.w[u][d] : 0.f;
  }

  long long f = fetch_trial(p.cursor, u == 0);
  f = __shfl_sync(kFull, f, root);
  bool active = f >= 0 && f < p.n;
  long long t = f;
  int k = 0;
  float s = 0.f, y = lg(0.f), netc = 0.f;
  // the noise of step k is drawn during step k - 1 (it does not depend on the
  // state), off the step's chain of shuffles and updates
  float e_next = 0.f;
  if (active && real) {
    netc = const_net(p, L.n_in, t, u);
    e_next = unit_noise(p, p.trial0 + (uint32_t)t, 0, L.U, u);
  }
  // phase 1 (EXT): the DDM nodes
  int phase = 0, net_step = 0;
  bool ddone = true;
  DdmNode dn{};
  int dchoice = -1, dstep = 0;
  float dx = 0.f;
  while (__any_sync(kFull, active)) {
    bool finished = false;
    if (active && (!EXT || phase == 0)) {
      // synchronous: every lane reads the step k outputs before any update
      float net = netc;
#pragma unroll
      for (int d = 0; d < kEdgeRegs; ++d) {
        if (d < D) {
          const float yv = __shfl_sync(gmask, y, root + esrc[d]);
          if (real) net = fmaf(ew[d], yv, net);
        }
      }
      for (int d = kEdgeRegs; d < D; ++d) {
        const int si = real ? L.src[u][d] : 0;
        const float yv = __shfl_sync(gmask, y, root + si);
        if (real) net = fmaf(L.w[u][d], yv, net);
      }
      if (real) {
        const float e = e_next;
        e_next = unit_noise(p, p.trial0 + (uint32_t)t, k + 1, L.U, u);
        s = fmaf(keep, s, fmaf(rate, net, noise * e));
        y = lg(s);
      }
      // top-1 (lowest index on ties) and top-2 of the stop layer
      float v1 = in_stop ? y : -FLT_MAX, v2 = -FLT_MAX;
      int i1 = in_stop ? u - stop_off : 1 << 20;
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
      const bool hit = v1 - v2 > thr;
      if (hit || k >= max_steps) {
        if (p.yout && in_stop) p.yout[(size_t)t * p.state_size + (u - stop_off)] = y;
        if (!EXT || L.n_ddm == 0) {
          if (u == 0) {
            p.choice[t] = hit ? (int8_t)i1 : (int8_t)-1;
            p.step[t] = hit ? k : L.max_steps;
          }
          finished = true;
        } else {
          // drifts of the DDM nodes from the stop layer's outputs
          net_step = hit ? k : L.max_steps;
          float drift = u < L.n_ddm ? L.ddm_bias[u] : 0.f;
          for (int i = 0; i < L.stop_size; ++i) {
            const float yi = __shfl_sync(gmask, y, root + L.stop_off + i);
            if (u < L.n_ddm) drift = fmaf(L.ddm_w[u][i], yi, drift);
          }
          ddone = u >= L.n_ddm;
          if (!ddone) dn = ddm_node_begin(L, u, drift);
          phase = 1;
        }
      }
    } else if (EXT && active) {
      if (!ddone) ddone = ddm_node_block(p, p.trial0 + (uint32_t)t, u, dn, dchoice, dstep, dx);
      if ((__ballot_sync(gmask, !ddone) & gmask) == 0u) {
        int cs[kNetMaxDdm], ss[kNetMaxDdm];
        for (int q = 0; q < L.n_ddm; ++q) {
          cs[q] = __shfl_sync(gmask, dchoice, root + q);
          ss[q] = __shfl_sync(gmask, dstep, root + q);
        }
        if (u == 0) ddm_response(L, cs, ss, net_step, p.choice[t], p.step[t]);
        if (p.yout && u < L.n_ddm) {
          float* o = p.yout + (size_t)t * p.state_size + L.stop_size + 3 * u;
          o[0] = dx;
          o[1] = (float)dchoice;
          o[2] = (float)dstep;
        }
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
      netc = (active && real) ? const_net(p, L.n_in, t, u) : 0.f;
      if (active && real) e_next = unit_noise(p, p.trial0 + (uint32_t)t, 0, L.U, u);
      phase = 0;
      ddone = true;
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
    netc[u * B + tid] = const_net(p, L.n_in, t, u);
    s[u * B + tid] = 0.f;
    y[u * B + tid] = Logistic::of(L.gain[u], L.bias[u])(0.f);
  }
  const uint32_t trial = p.trial0 + (uint32_t)t;
  bool hit = false;
  int best = 0, k = 0;
  const float* ys = y + L.stop_off * B + tid;
  while (k < L.max_steps) {
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int u = 0; u < U; ++u) {
      float net = netc[u * B + tid];
      for (int d = 0; d < L.D; ++d) net = fmaf(L.w[u][d], y[L.src[u][d] * B + tid], net);
      // the same normal as unit_noise, reusing a block across consecutive units
      const uint32_t dn = (uint32_t)k * (uint32_t)U + (uint32_t)u;
      if (u == 0 || (dn & 3u) == 0u) z = normals4(noise_block_rk(p.rk, trial, 0u, dn >> 2));
      const float e = pick4(z, dn & 3u);
      const float sv = fmaf(1.0f - L.rate, s[u * B + tid], fmaf(L.rate, net, L.noise * e));
      s[u * B + tid] = sv;
      yn[u * B + tid] = Logistic::of(L.gain[u], L.bias[u])(sv);
    }
    float* tmp = y;
    y = yn;
    yn = tmp;
    ys = y + L.stop_off * B + tid;
    ++k;
    best = 0;
    float v1 = ys[0];
    for (int i = 1; i < L.stop_size; ++i)
      if (ys[i * B] > v1) {
        v1 = ys[i * B];
        best = i;
      }
    float v2 = -FLT_MAX;
    for (int i = 0; i < L.stop_size; ++i)
      if (i != best) v2 = fmaxf(v2, ys[i * B]);
    hit = v1 - v2 > L.stop_threshold;
    if (hit) break;
  }
  const int net_step = hit ? k : L.max_steps;
  if (p.yout)
    for (int i = 0; i < L.stop_size; ++i) p.yout[(size_t)t * p.state_size + i] = ys[i * B];
  if (L.n_ddm == 0) {
    p.choice[t] = hit ? (int8_t)best : (int8_t)-1;
    p.step[t] = net_step;
    return;
  }
  int cs[kNetMaxDdm], ss[kNetMaxDdm];
  for (int q = 0; q < L.n_ddm; ++q) {
    float drift = L.ddm_bias[q];
    for (int i = 0; i < L.stop_size; ++i) drift = fmaf(L.ddm_w[q][i], ys[i * B], drift);
    DdmNode dn = ddm_node_begin(L, q, drift);
    float dx = 0.f;
    while (!ddm_node_block(p, trial, q, dn, cs[q], ss[q], dx)) {
    }
    if (p.yout) {
      float* o = p.yout + (size_t)t * p.state_size + L.stop_size + 3 * q;
      o[0] = dx;
      o[1] = (float)cs[q];
      o[2] = (float)ss[q];
    }
  }
  ddm_response(L, cs, ss, net_step, p.choice[t], p.step[t]);
}

size_t layout_smem() { return ((sizeof(NetLayout) + 15) / 16) * 16; }

template <int G, bool EXT>
cudaError_t launch_group(const NetParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  const size_t smem = layout_smem();
  cudaError_t e = smem_limit((const void*)net_group<G, EXT>, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, net_group<G, EXT>, 256, smem);
  if (nb < 1) nb = 1;
  long long grid = cfg.grid > 0 ? cfg.grid : (long long)num_sms() * nb;
  const long long need = (p.n * G + 255) / 256;
  if (grid > need) grid = need;
  net_group<G, EXT><<<(unsigned)grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_net(const NetParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  if (mode == 1 || p.cursor == nullptr) {
    const int B = 128;
    const size_t smem = layout_smem() + (size_t)4 * p.U * B * sizeof(float);
    cudaError_t e = smem_limit((const void*)net_plain, 200 * 1024);
    if (e != cudaSuccess) return e;
    net_plain<<<(unsigned)((p.n + B - 1) / B), B, smem, s>>>(p);
    return cudaGetLastError();
  }
  const int lanes = p.U > p.n_ddm ? p.U : p.n_ddm;   // a lane per unit and per DDM node
  if (p.n_ddm > 0) {
    if (lanes <= 8) return launch_group<8, true>(p, cfg, s);
    if (lanes <= 16) return launch_group<16, true>(p, cfg, s);
    return launch_group<32, true>(p, cfg, s);
  }
  if (lanes <= 2) return launch_group<2, false>(p, cfg, s);
  if (lanes <= 4) return launch_group<4, false>(p, cfg, s);
  if (lanes <= 8) return launch_group<8, false>(p, cfg, s);
  if (lanes <= 16) return launch_group<16, false>(p, cfg, s);
  return launch_group<32, false>(p, cfg, s);
}

}  // namespace dg
