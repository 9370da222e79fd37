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

__device__ __forceinline__ float const_net(const NetParams& p, int n_in, long long t, int u) {
  const long long g = (long long)p.trial0 + t;  // global trial id
  const int cond = (int)((g / p.cond_block) % p.n_cond);
  const float* cin = p.cond + (size_t)cond * n_in;
  const float* w = p.w_in + (size_t)u * n_in;
  float acc = 0.f;
  for (int q = 0; q < n_in; ++q) acc = fmaf(__ldg(w + q), __ldg(cin + q), acc);
  return acc;
}

__device__ __forceinline__ void stage_layout(const NetParams& p, unsigned char* smem) {
  const int words = (int)(sizeof(NetLayout) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(p.layout);
  uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

struct DdmNode {
  float adt, diff, z;
  int max;
  long long X;      // state before block b, fixed point
  int b;
};

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

// ---------------------------------------------------------- lane form ---

// One lane per trial (U <= kLaneMaxU units, no DDM nodes): the units' states
// and outputs in the lane's registers, the dense edge matrix read from the
// kernel parameters as instruction operands, and the normals of W steps (W U
// of them: whole Philox blocks, as W U is a multiple of 4) drawn together,
// the next window's while the current one runs. Each unit's incoming edges are
// sorted by sender, so the dense sum over senders adds the same nonzero terms
// in the same order as the edge table of the other forms (a zero term adds
// exactly nothing) and the lane form agrees with them bit for bit. A lane
// whose trial ends inside a window takes its next trial at the window's end,
// so that the lanes of a warp draw their noise together.
//
// SS > 0: the stop layer is the last SS units (known when compiling: the stop
// test and the kept outputs cover those units only); SS = 0: any range.
// MULTI: the trials of several jobs of the network (the serving loop's
// groups), one list over the jobs in order; a lane binds its trial's job
// (condition table, outputs, seed, trial offset) when it takes the trial on.
template <int U, int SS, bool MULTI>
__global__ void __launch_bounds__(128) net_lane(NetParams p, const __grid_constant__ NetDense q,
                                               const __grid_constant__
                                               typename TableOf<MULTI>::type tab) {
  __shared__ MultiJob s_job[MULTI ? kMaxMultiJobs : 1];
  if constexpr (MULTI) copy_jobs(tab, s_job);
  constexpr int W = (U % 2 == 0) ? 2 : 4;   // steps per window: W U normals in whole blocks
  constexpr int NZ = W * U;
  const float rate = q.rate, keep = 1.0f - q.rate, noise = q.noise, thr = q.thr;
  const int stop_off = SS > 0 ? U - SS : q.stop_off;
  const int stop_end = SS > 0 ? U : q.stop_off + q.stop_size;
  const int max_steps = q.max_steps;
  Logistic lg[U];
#pragma unroll
  for (int u = 0; u < U; ++u) lg[u] = Logistic::of(q.gain[u], q.bias[u]);
  float s[U], y[U], netc[U], z[NZ];
  long long t = 0;
  int k = 0;
  uint32_t trial = 0;
  NetParams pj = p;   // the lane's job: the launch's own, or bound from the table
  KeyPair kp{};
  // the normals of steps k0 .. k0 + W - 1 (k0 a multiple of W)
  auto draw = [&](int k0, float (&out)[NZ]) {
    const uint32_t b0 = (uint32_t)k0 * (uint32_t)U / 4u;
#pragma unroll
    for (int j = 0; j < NZ / 4; ++j) {
      uint4 w;
      if constexpr (MULTI)
        w = noise_block_rk(kp, trial, 0u, b0 + (uint32_t)j);
      else
        w = noise_block_rk(p.rk, trial, 0u, b0 + (uint32_t)j);
      const float4 v = normals4(w);
      out[4 * j] = v.x;
      out[4 * j + 1] = v.y;
      out[4 * j + 2] = v.z;
      out[4 * j + 3] = v.w;
    }
  };
  auto begin = [&](long long tt) {
    if constexpr (MULTI) {
      const MultiJob& J = s_job[multi_job_of(s_job, tab.n_jobs, tt)];
      pj.cond = J.in;
      pj.n_cond = J.n_cond;
      pj.cond_block = J.cond_block;
      pj.trial0 = J.trial0;
      pj.choice = J.choice;
      pj.step = J.step;
      pj.yout = J.xout;
      kp.k.k0 = J.k0;
      kp.k.k1 = J.k1;
      t = tt - J.start;
    } else {
      t = tt;
    }
    k = 0;
    trial = pj.trial0 + (uint32_t)t;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      s[u] = 0.f;
      y[u] = lg[u](0.f);
      netc[u] = const_net(pj, p.n_in, t, u);
    }
    draw(0, z);
  };
  long long f = fetch_trial(p.cursor, true);
  bool active = f >= 0 && f < p.n;
  if (active) begin(f);
  while (__any_sync(kFull, active)) {
    bool finished = false;
    if (active) {
      // two windows per iteration, the noise buffers in turn: while one
      // window's steps run, the next window's normals are drawn (independent
      // of the state). The steps run without branches (a trial that ends
      // inside the iteration runs on to its end, discarded) so that the
      // compiler can interleave them with the noise; the ending step's
      // results are kept by selects.
      int8_t rc = -1;
      int rs = 0;
      float ry[U];
#pragma unroll
      for (int u = 0; u < U; ++u) ry[u] = 0.f;
      auto steps = [&](const float (&zw)[NZ]) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          // synchronous: every net input from the previous step's outputs
          float net[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            float a = netc[u];
#pragma unroll
            for (int v = 0; v < U; ++v) a = fmaf(q.W[u][v], y[v], a);
            net[u] = a;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            s[u] = fmaf(keep, s[u], fmaf(rate, net[u], noise * zw[w * U + u]));
            y[u] = lg[u](s[u]);
          }
          ++k;
          // top-1 (lowest index on ties) and top-2 of the stop layer
          float v1 = -FLT_MAX, v2 = -FLT_MAX;
          int i1 = 1 << 20;
#pragma unroll
          for (int u = SS > 0 ? U - SS : 0; u < U; ++u) {
            if (SS > 0 || (u >= stop_off && u < stop_end)) {
              const bool up = y[u] > v1;
              v2 = up ? v1 : fmaxf(v2, y[u]);
              i1 = up ? u - stop_off : i1;
              v1 = up ? y[u] : v1;
            }
          }
          const bool hit = v1 - v2 > thr;
          const bool ends = !finished && (hit || k >= max_steps);
          rc = ends ? (hit ? (int8_t)i1 : (int8_t)-1) : rc;
          rs = ends ? (hit ? k : max_steps) : rs;
#pragma unroll
          for (int u = SS > 0 ? U - SS : 0; u < U; ++u) ry[u] = ends ? y[u] : ry[u];
          finished = finished || ends;
        }
      };
      float zn[NZ];
      draw(k + W, zn);
      steps(z);
      draw(k + W, z);   // k advanced by W: the window after zn's
      steps(zn);
      if (finished) {
        if (pj.yout) {
#pragma unroll
          for (int u = SS > 0 ? U - SS : 0; u < U; ++u)
            if (SS > 0 || (u >= stop_off && u < stop_end))
              pj.yout[(size_t)t * p.state_size + (u - stop_off)] = ry[u];
        }
        pj.choice[t] = rc;
        pj.step[t] = rs;
      }
    }
    f = fetch_trial(p.cursor, finished);
    if (finished) {
      active = f < p.n;
      if (active) begin(f);
    }
  }
}

template <int U, int SS, bool MULTI>
cudaError_t launch_lane_us(const NetParams& p, const NetDense& q, const MultiJobTable* tab,
                           cudaStream_t s) {
  int nb = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, net_lane<U, SS, MULTI>, 128, 0);
  if (e != cudaSuccess) return e;
  // small jobs: blocks of one warp spread over the SMs (a lane's step is a
  // chain of a few hundred instructions; warps sharing a scheduler slow it)
  const int block = p.n <= (long long)num_sms() * 32 * 4 ? 32 : 128;
  long long grid = (long long)num_sms() * (nb > 0 ? nb : 1) * (128 / block);
  const long long need = (p.n + block - 1) / block;
  if (grid > need) grid = need;
  if constexpr (MULTI)
    net_lane<U, SS, true><<<(unsigned)grid, block, 0, s>>>(p, q, *tab);
  else
    net_lane<U, SS, false><<<(unsigned)grid, block, 0, s>>>(p, q, {});
  return cudaGetLastError();
}

template <int U, bool MULTI>
cudaError_t launch_lane_u(const NetParams& p, const NetDense& q, const MultiJobTable* tab,
                          cudaStream_t s) {
  if (q.stop_off + q.stop_size == U) {   // the stop layer is last
    if (q.stop_size == 2) return launch_lane_us<U, (U >= 2 ? 2 : 0), MULTI>(p, q, tab, s);
    if (q.stop_size == 3) return launch_lane_us<U, (U >= 3 ? 3 : 0), MULTI>(p, q, tab, s);
    if (q.stop_size == 4) return launch_lane_us<U, (U >= 4 ? 4 : 0), MULTI>(p, q, tab, s);
  }
  return launch_lane_us<U, 0, MULTI>(p, q, tab, s);
}

template <bool MULTI>
cudaError_t launch_lane(const NetParams& p, const NetDense& q, const MultiJobTable* tab,
                        cudaStream_t s) {
  switch (p.U) {
    case 1: return launch_lane_u<1, MULTI>(p, q, tab, s);
    case 2: return launch_lane_u<2, MULTI>(p, q, tab, s);
    case 3: return launch_lane_u<3, MULTI>(p, q, tab, s);
    case 4: return launch_lane_u<4, MULTI>(p, q, tab, s);
    case 5: return launch_lane_u<5, MULTI>(p, q, tab, s);
    case 6: return launch_lane_u<6, MULTI>(p, q, tab, s);
    case 7: return launch_lane_u<7, MULTI>(p, q, tab, s);
    case 8: return launch_lane_u<8, MULTI>(p, q, tab, s);
  }
  return cudaErrorInvalidValue;
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

cudaError_t launch_net_lane(const NetParams& p, const NetDense& q, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  if (p.n_ddm != 0 || p.cursor == nullptr) return cudaErrorInvalidValue;
  return launch_lane<false>(p, q, nullptr, s);
}

cudaError_t launch_net_lane_multi(const NetParams& p, const NetDense& q, const MultiJobTable& tab,
                                  cudaStream_t s) {
  if (p.n <= 0 || tab.n_jobs < 1 || tab.n_jobs > kMaxMultiJobs) return cudaErrorInvalidValue;
  if (p.n_ddm != 0 || p.cursor == nullptr) return cudaErrorInvalidValue;
  return launch_lane<true>(p, q, &tab, s);
}

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
