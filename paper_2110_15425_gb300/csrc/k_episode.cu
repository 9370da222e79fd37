// Time-stepped predator-prey episodes (Sec. 2.1: the search over attention
// allocations is repeated at every time step until the prey or the player is
// caught; the positions carried from step to step are the sequential outer
// state that caps the parallelism of such models).
//
// Episode e keeps its positions S = (P, D, Y) in device memory. Step t:
//   - every allocation c is simulated on n_trials perceptions of S (noise
//     stream (trial t n_trials + j, cand c), Philox blocks 2e and 2e + 1, e
//     the global episode index), FP64 mean, best = argmax (lowest index on
//     ties);
//   - the player perceives S once more with the best allocation (stream
//     (trial t, cand 0xFFFFFFFF)) and moves speed[0] act; the predator steps
//     speed[1] unit(P - D) toward it, the prey speed[2] unit(Y - P) away, all
//     from the positions at the start of the step (this step runs in FP64 and
//     rounds the new positions to FP32);
//   - with the new positions, |P - Y| <= radius ends the episode with +1, else
//     |P - D| <= radius with -1; after T steps, 0.
//
// One launch per step over all episodes still running: the work is the list
// of (active episode, chunk of 64 candidates) pairs, taken in order by
// persistent blocks from an atomic cursor; each chunk's top-2 goes to a per-episode slot, and the
// block that completes an episode's last chunk merges them, moves the
// entities and appends the episode to the next step's list if it goes on.
// Three rotating lists: step t reads list t mod 3, appends to (t + 1) mod 3
// and clears (t + 2) mod 3, which nothing touches during step t.
#include "dg_device.cuh"
#include "dg_grid.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

// The move of the player, predator and prey is computed once per episode and
// step, by one thread, in FP64 with every operation rounded as written (no
// contraction), so the positions carried across steps stay as exact as their
// FP32 format allows.
__device__ __forceinline__ void unit2_f64(double vx, double vy, double& ox, double& oy) {
  const double n = __dsqrt_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)));
  if (n > 0.0) {
    ox = __ddiv_rn(vx, n);
    oy = __ddiv_rn(vy, n);
  } else {
    ox = 0.0;
    oy = 0.0;
  }
}

// Box-Muller pair in FP64 from words (wa, wb).
__device__ __forceinline__ void box_muller_f64(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  const double two_pi = 6.283185307179586476925286766559;
  const double ua = __dmul_rn(__dadd_rn((double)(wa >> 9), 0.5), 1.0 / 8388608.0);
  const double ub = __dmul_rn(__dadd_rn((double)(wb >> 9), 0.5), 1.0 / 8388608.0);
  const double r = __dsqrt_rn(__dmul_rn(-2.0, log(ua)));
  double sn, cs;
  sincos(__dmul_rn(two_pi, ub), &sn, &cs);
  z0 = __dmul_rn(r, cs);
  z1 = __dmul_rn(r, sn);
}

__global__ void episode_init(EpisodeParams p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p.E) {
    for (int d = 0; d < 6; ++d) p.state[6 * i + d] = p.start[6 * i + d];
    p.active[i] = i;
    p.ticket[i] = 0u;
    p.outcome[i] = 0;
    p.steps[i] = p.T;
    for (int t = 0; t < p.T; ++t) {
      if (p.traj_best) p.traj_best[(size_t)i * p.T + t] = -1;
      if (p.traj_value) p.traj_value[(size_t)i * p.T + t] = 0.0;
      if (p.traj_pos)
        for (int d = 0; d < 6; ++d) p.traj_pos[((size_t)i * p.T + t) * 6 + d] = 0.f;
    }
  }
  if (i == 0) {
    p.count[0] = p.E;
    p.count[1] = 0;
    p.count[2] = 0;
    for (int k = 0; k < 3; ++k) p.cursor[k] = 0ull;
  }
}

// Merge the episode's chunk summaries, move the entities, test for capture.
// Merge the episode's chunk summaries, move the entities, test for capture.
// The move runs on warp 0: lanes 0-2 draw and apply the perception noise of
// player, predator and prey (normal pair k of the step's stream is entity
// k's), lanes 3-4 the predator's and prey's directions, lanes 0-1 the two
// unit vectors of the Action node, lane 0 the rest.
__device__ void finish_episode(const EpisodeParams& p, int e) {
  __shared__ TopTwo warp_best[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TopTwo t = top_init();
  for (int b = threadIdx.x; b < p.cpe; b += blockDim.x) {
    const TopTwo* q = p.partials + (size_t)e * p.cpe + b;
    TopTwo v;
    v.v1 = __ldcg(&q->v1);
    v.i1 = __ldcg(&q->i1);
    v.v2 = __ldcg(&q->v2);
    t = top_merge(t, v);
  }
  t = top_warp(t);
  if (lane == 0) warp_best[warp] = t;
  __syncthreads();
  if (warp != 0) return;
  TopTwo r = warp_best[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = top_merge(r, warp_best[w]);
  const long long b = r.i1;
  const int l2 = (int)(b % p.L[2]);
  const int l1 = (int)((b / p.L[2]) % p.L[1]);
  const int l0 = (int)(b / ((long long)p.L[2] * p.L[1]));
  float S[6];
  for (int d = 0; d < 6; ++d) S[d] = __ldcg(p.state + 6 * e + d);
  double mx = 0.0, my = 0.0;
  if (lane < 3) {
    // perceived position of entity `lane` with the chosen allocation
    const float a = lane == 0 ? p.lv[0][l0] : (lane == 1 ? p.lv[1][l1] : p.lv[2][l2]);
    const uint4 w = noise_block_rk(p.rk, (uint32_t)p.t, 0xFFFFFFFFu,
                                2u * (p.e0 + (uint32_t)e) + (lane == 2 ? 1u : 0u));
    double z0, z1;
    box_muller_f64(lane == 1 ? w.z : w.x, lane == 1 ? w.w : w.y, z0, z1);
    const double sd = __ddiv_rn(1.0, __dadd_rn(p.offset_d, (double)a));
    mx = __dadd_rn((double)S[2 * lane], __dmul_rn(sd, z0));
    my = __dadd_rn((double)S[2 * lane + 1], __dmul_rn(sd, z1));
  } else if (lane == 3) {  // the predator pursues the player
    unit2_f64(__dsub_rn((double)S[0], (double)S[2]), __dsub_rn((double)S[1], (double)S[3]), mx,
              my);
  } else if (lane == 4) {  // the prey flees it
    unit2_f64(__dsub_rn((double)S[4], (double)S[0]), __dsub_rn((double)S[5], (double)S[1]), mx,
              my);
  }
  const double ppx = __shfl_sync(kFull, mx, 0), ppy = __shfl_sync(kFull, my, 0);
  const double pdx = __shfl_sync(kFull, mx, 1), pdy = __shfl_sync(kFull, my, 1);
  const double pyx = __shfl_sync(kFull, mx, 2), pyy = __shfl_sync(kFull, my, 2);
  const double ux = __shfl_sync(kFull, mx, 3), uy = __shfl_sync(kFull, my, 3);
  const double vx = __shfl_sync(kFull, mx, 4), vy = __shfl_sync(kFull, my, 4);
  double qx = 0.0, qy = 0.0;
  if (lane == 0) unit2_f64(__dsub_rn(pyx, ppx), __dsub_rn(pyy, ppy), qx, qy);
  if (lane == 1) unit2_f64(__dsub_rn(pdx, ppx), __dsub_rn(pdy, ppy), qx, qy);
  const double udx = __shfl_sync(kFull, qx, 1), udy = __shfl_sync(kFull, qy, 1);
  if (lane != 0) return;
  double ax, ay;
  unit2_f64(__dsub_rn(qx, __dmul_rn(p.weight_d, udx)), __dsub_rn(qy, __dmul_rn(p.weight_d, udy)),
            ax, ay);
  float N[6];
  N[0] = __double2float_rn(__dadd_rn((double)S[0], __dmul_rn(p.speed[0], ax)));
  N[1] = __double2float_rn(__dadd_rn((double)S[1], __dmul_rn(p.speed[0], ay)));
  N[2] = __double2float_rn(__dadd_rn((double)S[2], __dmul_rn(p.speed[1], ux)));
  N[3] = __double2float_rn(__dadd_rn((double)S[3], __dmul_rn(p.speed[1], uy)));
  N[4] = __double2float_rn(__dadd_rn((double)S[4], __dmul_rn(p.speed[2], vx)));
  N[5] = __double2float_rn(__dadd_rn((double)S[5], __dmul_rn(p.speed[2], vy)));
  for (int d = 0; d < 6; ++d) p.state[6 * e + d] = N[d];
  const size_t k = (size_t)e * p.T + p.t;
  if (p.traj_best) p.traj_best[k] = (int32_t)b;
  if (p.traj_value) p.traj_value[k] = r.v1;
  if (p.traj_pos)
    for (int d = 0; d < 6; ++d) p.traj_pos[k * 6 + d] = N[d];
  const double cyx = __dsub_rn((double)N[0], (double)N[4]);
  const double cyy = __dsub_rn((double)N[1], (double)N[5]);
  const double cdx = __dsub_rn((double)N[0], (double)N[2]);
  const double cdy = __dsub_rn((double)N[1], (double)N[3]);
  int8_t out = 0;
  bool done = false;
  if (__dsqrt_rn(__dadd_rn(__dmul_rn(cyx, cyx), __dmul_rn(cyy, cyy))) <= p.radius) {
    out = 1;
    done = true;
  } else if (__dsqrt_rn(__dadd_rn(__dmul_rn(cdx, cdx), __dmul_rn(cdy, cdy))) <= p.radius) {
    out = -1;
    done = true;
  }
  if (p.t + 1 >= p.T) done = true;
  if (done) {
    p.outcome[e] = out;
    p.steps[e] = p.t + 1;
    if (p.final_pos)
      for (int d = 0; d < 6; ++d) p.final_pos[6 * e + d] = N[d];
  } else {
    int* next = p.active + (size_t)((p.t + 1) % 3) * p.E;
    next[atomicAdd(p.count + (p.t + 1) % 3, 1)] = e;
  }
  p.ticket[e] = 0u;  // ready for the next step
}

// LANES lanes per candidate, as the grid search takes them for a grid of this
// size (grid_lanes): eight, four candidates per warp, for grids of 16,384
// candidates or more, else a whole warp.
template <int LANES>
__global__ void __launch_bounds__(256) episode_step(EpisodeParams p) {
  constexpr int kPerWarp = 32 / LANES;   // candidates of a warp at a time
  __shared__ TopTwo warp_best[8];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ long long item;
  const int cur = p.t % 3;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.count[(p.t + 2) % 3] = 0;
    p.cursor[(p.t + 2) % 3] = 0ull;
  }
  const int na = __ldcg(p.count + cur);
  const int* act = p.active + (size_t)cur * p.E;
  const long long items = (long long)na * p.cpe;
  const double inv = 1.0 / (double)p.n_trials;
  const uint32_t trial0 = (uint32_t)p.t * (uint32_t)p.n_trials;
  for (;;) {
    // items are taken in order from the step's cursor, so a block that
    // finishes an episode does not hold up the items after it
    if (threadIdx.x == 0) item = (long long)atomicAdd(p.cursor + cur, 1ull);
    __syncthreads();
    const long long w = item;
    if (w >= items) break;
    const int e = __ldcg(act + w / p.cpe);
    const int chunk = (int)(w % p.cpe);
    float S[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) S[d] = __ldcg(p.state + 6 * e + d);
    TopTwo best = top_init();
    const long long c_end = min((long long)(chunk + 1) * kEpisodeChunk, p.n_cand);
    // the block's 64 candidates, kPerWarp per warp at a time: group g of warp w
    // takes candidate c0 + 8 kPerWarp i + kPerWarp w + g; lane kPerWarp i + g
    // keeps its pair, and the warp's means are formed in FP64 together at the end
    const int grp = lane / LANES, gl = lane % LANES;
    const long long c0 = (long long)chunk * kEpisodeChunk;
    float kh = 0.f, kl = 0.f;
    long long kc = -1;
    for (int i = 0; (long long)i * 8 * kPerWarp < kEpisodeChunk; ++i) {
      const long long cb = c0 + (long long)i * 8 * kPerWarp + (long long)warp * kPerWarp;
      const long long c = cb + grp;
      float hi = 0.f, lo = 0.f;
      if (c < c_end) {
        const uint32_t u = (uint32_t)c, q = u / (uint32_t)p.L[2];   // c < 2^32 (n_cand checked)
        const int l2 = (int)(u - q * (uint32_t)p.L[2]);
        const int l1 = (int)(q % (uint32_t)p.L[1]);
        const int l0 = (int)(q / (uint32_t)p.L[1]);
        const float a0 = __ldg(p.lv[0] + l0), a1 = __ldg(p.lv[1] + l1), a2 = __ldg(p.lv[2] + l2);
        const float sd0 = 1.0f / (p.offset + a0), sd1 = 1.0f / (p.offset + a1),
                    sd2 = 1.0f / (p.offset + a2);
        const float cost = a0 * a0 + a1 * a1 + a2 * a2;
        for (int j = gl; j < p.n_trials; j += LANES)
          two_sum_add(hi, lo, pp_outcome_at(p.rk, trial0 + (uint32_t)j, (uint32_t)c,
                                            2u * (p.e0 + (uint32_t)e), S, sd0, sd1, sd2,
                                            p.weight, cost));
      }
      group_pair_sum<LANES>(hi, lo);
      const int g = lane - i * kPerWarp;
      const bool mine = g >= 0 && g < kPerWarp;
      const int src = mine ? g * LANES : 0;
      const float th = __shfl_sync(kFull, hi, src), tl = __shfl_sync(kFull, lo, src);
      if (mine && cb + g < c_end) {
        kh = th;
        kl = tl;
        kc = cb + g;
      }
    }
    if (kc >= 0) best = TopTwo{pair_mean(kh, kl, inv), kc, -DBL_MAX};
    best = top_warp(best);
    if (lane == 0) warp_best[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      TopTwo r = warp_best[0];
      for (int i = 1; i < 8; ++i) r = top_merge(r, warp_best[i]);
      p.partials[(size_t)e * p.cpe + chunk] = r;
      __threadfence();
      last = atomicAdd(p.ticket + e, 1u) == (unsigned)(p.cpe - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      finish_episode(p, e);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_episode_init(const EpisodeParams& p, cudaStream_t s) {
  episode_init<<<(p.E + 255) / 256, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_episode_step(const EpisodeParams& p, cudaStream_t s) {
  const bool narrow = grid_lanes(p.L) == 8;
  // resident blocks of the current device (asked per launch: a process may
  // drive GPUs of different sizes)
  int nb = 0;
  const cudaError_t e =
      narrow ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, episode_step<8>, 256, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, episode_step<32>, 256, 0);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)num_sms() * (nb > 0 ? nb : 1);
  long long g = (long long)p.E * p.cpe;
  if (g > blocks) g = blocks;
  if (narrow)
    episode_step<8><<<(unsigned)g, 256, 0, s>>>(p);
  else
    episode_step<32><<<(unsigned)g, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace dg
