// Small networks, one lane per trial (kernel templates; each k_net_lane*.cu
// file instantiates one variant, so that they compile in parallel) (the Botvinick Stroop model of Sec. 5 and
// the Extended Stroop's DDM nodes): the batched form for networks of at most
// kLaneMaxU logistic units. Every unit integrates with time averaging,
//   s <- (1 - rate) s + rate net + noise eps,  y = 1 / (1 + exp(-gain (s + bias))),
// all units read the previous iteration's outputs (synchronous update), and a
// trial ends at the first step where the stop layer's largest output exceeds
// the second largest by more than the threshold; then its DDM nodes, if any,
// integrate x += drift dt + sigma sqrt(dt) eps from 0 to a bound (FP32 sums
// within each 4-step Philox block, 64-bit fixed point across blocks). The
// arithmetic is the lane-group and plain forms' (k_net.cu), term for term.
#pragma once

#include <cfloat>

#include "dg_device.cuh"
#include "dg_internal.h"
#include "dg_net.cuh"

namespace dg {

namespace {

// One block (4 steps) of a node with its normals e, the arithmetic of the
// lane-group and plain forms' node blocks (k_net.cu); true when the node has
// ended.
__device__ __forceinline__ bool ddm_node_step4(DdmNode& d, const float4& e, int& choice,
                                               int& step, float& x) {
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

// The whole of node q in one lane, block after block, with each block's
// normals drawn while the block before it is tested (they do not
// depend on the state), so that the Philox and Box-Muller chain overlaps the
// sums and bound tests.
__device__ __forceinline__ void ddm_node_lane(const NetParams& p, uint32_t trial, int q,
                                              DdmNode d, int& choice, int& step, float& x) {
  float4 e = normals4(noise_block_rk(p.rk, trial, 1u + (uint32_t)q, (uint32_t)d.b));
  while (true) {
    const float4 en = normals4(noise_block_rk(p.rk, trial, 1u + (uint32_t)q, (uint32_t)d.b + 1u));
    if (ddm_node_step4(d, e, choice, step, x)) return;
    e = en;
  }
}

// ---------------------------------------------------------- lane form ---

// One lane per trial (U <= kLaneMaxU units): the units' states
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
// EXT: the network's DDM nodes run after it, in the same lane (one job only).
template <int U, int SS, bool MULTI, bool EXT>
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
        if constexpr (!EXT) {
          pj.choice[t] = rc;
          pj.step[t] = rs;
        } else {
          // the DDM nodes, in order, in this lane (as the plain form runs them):
          // drift_n = bias_n + sum_i w_ni y_i over the stop layer in unit
          // order; the response is the node that decides in the fewest steps
          // (the lower node on equal steps)
          int best = -1, best_c = 0, best_s = 0, longest = 0;
          auto node = [&](int n) {
            float drift = q.ddm_bias[n];
#pragma unroll
            for (int u = SS > 0 ? U - SS : 0; u < U; ++u)
              if (SS > 0 || (u >= stop_off && u < stop_end))
                drift = fmaf(q.ddm_w[n][u - stop_off], ry[u], drift);
            return DdmNode{drift * q.ddm_dt[n], q.ddm_diffusion[n], q.ddm_z[n], q.ddm_max[n], 0ll,
                           0};
          };
          auto done = [&](int n, int c, int st, float xn) {
            if (pj.yout) {
              float* o = pj.yout + (size_t)t * p.state_size + q.stop_size + 3 * n;
              o[0] = xn;
              o[1] = (float)c;
              o[2] = (float)st;
            }
            if (c >= 0 && (best < 0 || st < best_s)) {
              best = n;
              best_c = c;
              best_s = st;
            }
            longest = max(longest, q.ddm_max[n]);
          };
          for (int n = 0; n < q.n_ddm; ++n) {
            int c = -1, st = 0;
            float xn = 0.f;
            ddm_node_lane(p, trial, n, node(n), c, st, xn);
            done(n, c, st, xn);
          }
          pj.choice[t] = best >= 0 ? (int8_t)(2 * best + best_c) : (int8_t)-1;
          pj.step[t] = rs + (best >= 0 ? best_s : longest);
        }
      }
    }
    f = fetch_trial(p.cursor, finished);
    if (finished) {
      active = f < p.n;
      if (active) begin(f);
    }
  }
}

template <int U, int SS, bool MULTI, bool EXT>
cudaError_t launch_lane_us(const NetParams& p, const NetDense& q, const MultiJobTable* tab,
                           cudaStream_t s) {
  int nb = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, net_lane<U, SS, MULTI, EXT>, 128, 0);
  if (e != cudaSuccess) return e;
  // small jobs: blocks of one warp spread over the SMs (a lane's step is a
  // chain of a few hundred instructions; warps sharing a scheduler slow it)
  const int block = p.n <= (long long)num_sms() * 32 * 4 ? 32 : 128;
  long long grid = (long long)num_sms() * (nb > 0 ? nb : 1) * (128 / block);
  const long long need = (p.n + block - 1) / block;
  if (grid > need) grid = need;
  if constexpr (MULTI)
    net_lane<U, SS, true, false><<<(unsigned)grid, block, 0, s>>>(p, q, *tab);
  else
    net_lane<U, SS, false, EXT><<<(unsigned)grid, block, 0, s>>>(p, q, {});
  return cudaGetLastError();
}

template <int U, bool MULTI, bool EXT>
cudaError_t launch_lane_u(const NetParams& p, const NetDense& q, const MultiJobTable* tab,
                          cudaStream_t s) {
  if (q.stop_off + q.stop_size == U) {   // the stop layer is last
    if (q.stop_size == 2) return launch_lane_us<U, (U >= 2 ? 2 : 0), MULTI, EXT>(p, q, tab, s);
    if (q.stop_size == 3) return launch_lane_us<U, (U >= 3 ? 3 : 0), MULTI, EXT>(p, q, tab, s);
    if (q.stop_size == 4) return launch_lane_us<U, (U >= 4 ? 4 : 0), MULTI, EXT>(p, q, tab, s);
  }
  return launch_lane_us<U, 0, MULTI, EXT>(p, q, tab, s);
}

template <bool MULTI, bool EXT>
cudaError_t launch_lane(const NetParams& p, const NetDense& q, const MultiJobTable* tab,
                        cudaStream_t s) {
  switch (p.U) {
    case 1: return launch_lane_u<1, MULTI, EXT>(p, q, tab, s);
    case 2: return launch_lane_u<2, MULTI, EXT>(p, q, tab, s);
    case 3: return launch_lane_u<3, MULTI, EXT>(p, q, tab, s);
    case 4: return launch_lane_u<4, MULTI, EXT>(p, q, tab, s);
    case 5: return launch_lane_u<5, MULTI, EXT>(p, q, tab, s);
    case 6: return launch_lane_u<6, MULTI, EXT>(p, q, tab, s);
    case 7: return launch_lane_u<7, MULTI, EXT>(p, q, tab, s);
    case 8: return launch_lane_u<8, MULTI, EXT>(p, q, tab, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace dg
