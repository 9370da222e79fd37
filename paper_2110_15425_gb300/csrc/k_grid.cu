// Optimization-control grid search of the predator-prey model (Sec. 2.1,
// Fig. pp_eg; parallel evaluation of Sec. 3.6).
//
// Candidate c = (l0 L1 + l1) L2 + l2 allocates attention a = (lv0[l0], lv1[l1],
// lv2[l2]) to (player, predator, prey). Trial j of candidate c:
//   perceived X^_e = X_e + eps_{2e+coord} / (offset + a_e)   (stream (seed, j, c))
//   act = unit(unit(Y^ - P^) - weight unit(D^ - P^)),  unit(0) = 0
//   outcome = -|P + act - Y| - sum_e a_e^2                      (true P, Y)
// mean_c = FP64 mean of the outcomes; best = argmax_c mean_c, lowest c on ties.
//
// Batched form: a group of lanes per candidate (the trials spread over them;
// eight lanes, four candidates per warp, for grids of 16,384 candidates or
// more, else a whole warp), a compensated FP32 pair sum across the group
// converted to the FP64 mean, running top-2 per warp, block merge, then the
// last block to finish merges the per-block partials (no second launch, no
// atomics on the values). Plain form (the paper's mapping): one thread per candidate
// with a sequential FP64 sum, then a separate argmax launch.
//
// Random tie-break (Sec. 3.3: one of several equally good choices is picked at
// random by reservoir sampling). A one-element reservoir filled in candidate
// order (Vitter's Algorithm R) ends holding the last tie t_k, among the ties
// t_1 < t_2 < ... at the maximum, whose draw accepted its rank k (t_1 always
// does; t_k for k >= 2 when w k < 2^32, w = word 0 of Philox(seed, counter
// (t_k lo, t_k hi, 0, 4))). tie_reservoir computes exactly that after the
// argmax: one block scans the stored means in index order, ranks the ties by
// a block prefix count, and keeps the largest accepted index.
#include <cfloat>
#include <climits>

#include "dg_device.cuh"
#include "dg_grid.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

// c: the candidate's noise stream
__device__ __forceinline__ float pp_outcome(const GridParams& p, const float* pos, int j,
                                            uint32_t c, float sd0, float sd1, float sd2,
                                            float cost) {
  return pp_outcome_at(p.rk, (uint32_t)j, c, 0u, pos + 6 * j, sd0, sd1, sd2, p.weight, cost);
}

// c: global candidate index (32-bit division whenever c fits: the 64-bit
// forms are long software sequences)
__device__ __forceinline__ void cand_alloc(const GridParams& p, const float* lv, long long c,
                                           float& a0, float& a1, float& a2) {
  int l0, l1, l2;
  if ((unsigned long long)c <= 0xFFFFFFFFull) {
    const uint32_t u = (uint32_t)c, q = u / (uint32_t)p.L[2];
    l2 = (int)(u - q * (uint32_t)p.L[2]);
    l1 = (int)(q % (uint32_t)p.L[1]);
    l0 = (int)(q / (uint32_t)p.L[1]);
  } else {
    l2 = (int)(c % p.L[2]);
    l1 = (int)((c / p.L[2]) % p.L[1]);
    l0 = (int)(c / ((long long)p.L[2] * p.L[1]));
  }
  a0 = lv[l0];
  a1 = lv[p.L[0] + l1];
  a2 = lv[p.L[0] + p.L[1] + l2];
}

// Stage positions and level values in shared memory.
__device__ __forceinline__ void stage(const GridParams& p, float* pos, float* lv) {
  for (int i = threadIdx.x; i < 6 * p.n_trials; i += blockDim.x) pos[i] = __ldg(p.pos + i);
  for (int i = threadIdx.x; i < p.L[0]; i += blockDim.x) lv[i] = __ldg(p.lv[0] + i);
  for (int i = threadIdx.x; i < p.L[1]; i += blockDim.x) lv[p.L[0] + i] = __ldg(p.lv[1] + i);
  for (int i = threadIdx.x; i < p.L[2]; i += blockDim.x)
    lv[p.L[0] + p.L[1] + i] = __ldg(p.lv[2] + i);
  __syncthreads();
}

// Block-wide merge of per-warp summaries, publication of the block's summary,
// and the final merge by whichever block finishes last.
__device__ void finish_argmax(TopTwo mine, TopTwo* partials, unsigned int* ticket,
                              void* result) {
  __shared__ TopTwo warp_best[32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  mine = top_warp(mine);
  if (lane == 0) warp_best[warp] = mine;
  __syncthreads();
  if (warp == 0) {
    TopTwo t = lane < nw ? warp_best[lane] : top_init();
    t = top_warp(t);
    if (lane == 0) {
      partials[blockIdx.x] = t;
      __threadfence();
      last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  TopTwo t = top_init();
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    TopTwo q;
    q.v1 = __ldcg(&partials[b].v1);
    q.i1 = __ldcg(&partials[b].i1);
    q.v2 = __ldcg(&partials[b].v2);
    t = top_merge(t, q);
  }
  t = top_warp(t);
  __syncthreads();
  if (lane == 0) warp_best[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    TopTwo r = warp_best[0];
    for (int w = 1; w < nw; ++w) r = top_merge(r, warp_best[w]);
    GridResultDev* out = reinterpret_cast<GridResultDev*>(result);
    out->best_index = r.i1;
    out->best_value = r.v1;
    out->gap = (r.v2 == -DBL_MAX) ? 0.0 : r.v1 - r.v2;
  }
}

template <int LANES>
__global__ void __launch_bounds__(256) grid_batched(GridParams p) {
  constexpr int kGridLanes = LANES, kGridCandsPerWarp = 32 / LANES;
  extern __shared__ float sm[];
  float* pos = sm;
  float* lv = sm + 6 * p.n_trials;
  stage(p, pos, lv);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / kGridLanes, gl = lane % kGridLanes;
  const int wpb = blockDim.x >> 5;
  TopTwo best = top_init();
  const double inv = 1.0 / (double)p.n_trials;
  // lane `slot + g` keeps the pair of group g's candidate; every 32
  // candidates (and at the end) all lanes convert theirs to FP64 at once
  float kh = 0.f, kl = 0.f;
  long long kc = -1;
  int slot = 0;
  auto flush = [&]() {
    if (kc >= 0) {
      const double mean = pair_mean(kh, kl, inv);
      if (p.means) p.means[kc] = mean;
      best = top_merge(best, TopTwo{mean, p.cand0 + kc, -DBL_MAX});
    }
    kc = -1;
  };
  for (long long cb = ((long long)blockIdx.x * wpb + warp) * kGridCandsPerWarp; cb < p.n_cand;
       cb += (long long)gridDim.x * wpb * kGridCandsPerWarp) {
    const long long c = cb + grp;
    float hi = 0.f, lo = 0.f;
    if (c < p.n_cand) {
      const long long cg = p.cand0 + c;
      float a0, a1, a2;
      cand_alloc(p, lv, cg, a0, a1, a2);
      const float sd0 = 1.0f / (p.offset + a0), sd1 = 1.0f / (p.offset + a1),
                  sd2 = 1.0f / (p.offset + a2);
      const float cost = a0 * a0 + a1 * a1 + a2 * a2;
      for (int j = gl; j < p.n_trials; j += kGridLanes)
        two_sum_add(hi, lo, pp_outcome(p, pos, j, p.stream0 + (uint32_t)cg, sd0, sd1, sd2, cost));
    }
    group_pair_sum<LANES>(hi, lo);
    // lane slot + g takes group g's total from the group's first lane
    const int g = lane - slot;
    const bool mine = g >= 0 && g < kGridCandsPerWarp;
    const int src = mine ? g * kGridLanes : 0;
    const float th = __shfl_sync(kFull, hi, src), tl = __shfl_sync(kFull, lo, src);
    if (mine && cb + g < p.n_cand) {
      kh = th;
      kl = tl;
      kc = cb + g;
    }
    slot += kGridCandsPerWarp;
    if (slot == 32) {
      flush();
      slot = 0;
    }
  }
  flush();
  finish_argmax(best, p.partials, p.ticket, p.result);
}

__global__ void __launch_bounds__(256) grid_plain(GridParams p) {
  extern __shared__ float sm[];
  float* pos = sm;
  float* lv = sm + 6 * p.n_trials;
  stage(p, pos, lv);
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.n_cand) return;
  const long long cg = p.cand0 + c;
  float a0, a1, a2;
  cand_alloc(p, lv, cg, a0, a1, a2);
  const float sd0 = 1.0f / (p.offset + a0), sd1 = 1.0f / (p.offset + a1),
              sd2 = 1.0f / (p.offset + a2);
  const float cost = a0 * a0 + a1 * a1 + a2 * a2;
  double acc = 0.0;
  for (int j = 0; j < p.n_trials; ++j)
    acc += (double)pp_outcome(p, pos, j, p.stream0 + (uint32_t)cg, sd0, sd1, sd2, cost);
  p.means[c] = acc / (double)p.n_trials;
}

__global__ void __launch_bounds__(256) argmax_kernel(const double* v, long long n,
                                                     long long base, TopTwo* partials,
                                                     unsigned int* ticket, void* result) {
  TopTwo best = top_init();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    best = top_merge(best, TopTwo{v[i], base + i, -DBL_MAX});
  finish_argmax(best, partials, ticket, result);
}

// A batch of whole-grid searches (GridBatchParams): persistent blocks take
// (search, chunk of kGridChunk candidates) items in order from a cursor;
// each candidate is evaluated exactly as grid_batched does (the same lanes per
// candidate, trial split, pair sums and FP64 mean, so its mean has the same
// bits), the chunk's top-2 goes to the search's partials, and the block that
// completes a search's last chunk merges them into its result. Many searches
// per launch amortise the ramp and drain that a one-wave search pays.
template <int LANES>
__global__ void __launch_bounds__(256) grid_batch(GridBatchParams p) {
  constexpr int kPerWarp = 32 / LANES;
  __shared__ TopTwo warp_best[8];
  __shared__ bool last;
  __shared__ long long item;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / LANES, gl = lane % LANES;
  const long long items = (long long)p.n_search * p.cpc;
  const double inv = 1.0 / (double)p.n_trials;
  for (;;) {
    if (threadIdx.x == 0) item = (long long)atomicAdd(p.cursor, 1ull);
    __syncthreads();
    const long long w = item;
    if (w >= items) break;
    const int si = (int)(w / p.cpc);
    const int chunk = (int)(w % p.cpc);
    const GridBatchItem& S = p.items[si];
    const PhiloxKeys rk = philox_keys(S.k0, S.k1);
    const long long c0 = (long long)chunk * kGridChunk;
    const long long c_end = min(c0 + kGridChunk, p.n_cand);
    float kh = 0.f, kl = 0.f;
    long long kc = -1;
    for (int i = 0; i * 8 * kPerWarp < kGridChunk; ++i) {
      const long long cb = c0 + (long long)i * 8 * kPerWarp + (long long)warp * kPerWarp;
      const long long c = cb + grp;
      float hi = 0.f, lo = 0.f;
      if (c < c_end) {
        const uint32_t u = (uint32_t)c, q = u / (uint32_t)p.L[2];   // c < 2^32 (checked)
        const int l2 = (int)(u - q * (uint32_t)p.L[2]);
        const int l1 = (int)(q % (uint32_t)p.L[1]);
        const int l0 = (int)(q / (uint32_t)p.L[1]);
        const float a0 = __ldg(S.lv[0] + l0), a1 = __ldg(S.lv[1] + l1), a2 = __ldg(S.lv[2] + l2);
        const float sd0 = 1.0f / (p.offset + a0), sd1 = 1.0f / (p.offset + a1),
                    sd2 = 1.0f / (p.offset + a2);
        const float cost = a0 * a0 + a1 * a1 + a2 * a2;
        for (int j = gl; j < p.n_trials; j += LANES) {
          float X[6];
#pragma unroll
          for (int d = 0; d < 6; ++d) X[d] = __ldg(S.pos + 6 * j + d);
          two_sum_add(hi, lo, pp_outcome_at(rk, (uint32_t)j, (uint32_t)c, 0u, X, sd0, sd1, sd2,
                                            p.weight, cost));
        }
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
    TopTwo best = top_init();
    if (kc >= 0) {
      const double mean = pair_mean(kh, kl, inv);
      if (S.means) S.means[kc] = mean;
      best = TopTwo{mean, kc, -DBL_MAX};
    }
    best = top_warp(best);
    if (lane == 0) warp_best[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      TopTwo r = warp_best[0];
      for (int i = 1; i < 8; ++i) r = top_merge(r, warp_best[i]);
      p.partials[(size_t)si * p.cpc + chunk] = r;
      __threadfence();
      last = atomicAdd(p.ticket + si, 1u) == (unsigned)(p.cpc - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      TopTwo t = top_init();
      for (int b = threadIdx.x; b < p.cpc; b += blockDim.x) {
        const TopTwo* q = p.partials + (size_t)si * p.cpc + b;
        TopTwo v;
        v.v1 = __ldcg(&q->v1);
        v.i1 = __ldcg(&q->i1);
        v.v2 = __ldcg(&q->v2);
        t = top_merge(t, v);
      }
      t = top_warp(t);
      if (lane == 0) warp_best[warp] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        TopTwo r = warp_best[0];
        for (int i = 1; i < 8; ++i) r = top_merge(r, warp_best[i]);
        GridResultDev* out = reinterpret_cast<GridResultDev*>(S.result);
        out->best_index = r.i1;
        out->best_value = r.v1;
        out->gap = (r.v2 == -DBL_MAX) ? 0.0 : r.v1 - r.v2;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool reservoir_accepts(uint32_t k0, uint32_t k1, long long i,
                                                  long long k) {
  if (k == 1) return true;
  const unsigned long long u = (unsigned long long)i;
  const uint4 w = philox(make_uint4((uint32_t)u, (uint32_t)(u >> 32), 0u, 4u), k0, k1);
  return (unsigned long long)w.x * (unsigned long long)k < (1ull << 32);
}

__global__ void __launch_bounds__(1024) tie_reservoir(const double* v, long long n,
                                                      long long base, uint32_t k0,
                                                      uint32_t k1, void* result) {
  __shared__ int cnt[32];
  __shared__ long long pick[32];
  GridResultDev* out = reinterpret_cast<GridResultDev*>(result);
  const double top = out->best_value;
  // gap != 0: the maximum is unique and the argmax already holds it
  if (n < 2 || out->gap != 0.0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  long long rank0 = 0, chosen = -1;
  for (long long start = 0; start < n; start += blockDim.x) {
    const long long i = start + threadIdx.x;
    const bool tie = i < n && v[i] == top;
    const unsigned b = __ballot_sync(kFull, tie);
    if (lane == 0) cnt[warp] = __popc(b);
    __syncthreads();
    int before = __popc(b & ((1u << lane) - 1u)), total = 0;
    for (int w = 0; w < nw; ++w) {
      total += cnt[w];
      if (w < warp) before += cnt[w];
    }
    if (tie && reservoir_accepts(k0, k1, base + i, rank0 + before + 1)) chosen = base + i;
    rank0 += total;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(kFull, chosen, o);
    chosen = other > chosen ? other : chosen;
  }
  if (lane == 0) pick[warp] = chosen;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long c = pick[0];
    for (int w = 1; w < nw; ++w) c = pick[w] > c ? pick[w] : c;
    if (c >= 0) out->best_index = c;
  }
}

// ------------------------------------------------- coarse-to-fine grid ---
// The search-space refinement of Sec. 4.3, by simulation: round r lays G
// points on each signal's interval, level l = lo + (hi - lo) l / (G - 1)
// (FP64, rounded to FP32), simulates the G^3 candidates with noise streams
// r G^3 + c (grid_batched with stream0 = r G^3), and centres the next
// interval on the best level with half-width one grid spacing, clipped to the
// domain. The explicit _rn intrinsics keep the FP64 steps unfused, as the
// definition states them.

struct RefineRoundDev {          // dg_refine_round
  float alloc[3];
  float lo[3];
  float hi[3];
  int round;
  long long best_index;          // this and the next two: a dg_grid_result
  double value;
  double gap;
};
static_assert(sizeof(RefineRoundDev) == 64, "dg_refine_round layout");

// x / (G - 1), correctly rounded. A power-of-two divisor has an exact
// reciprocal, and the product then rounds exactly as the quotient does; the
// double-precision divide, a long sequence on this GPU, is left for other G.
__device__ __forceinline__ double div_g1(double x, int G) {
  const int d = G - 1;
  if ((d & (d - 1)) == 0) {
    const long long k = __ffs(d) - 1;   // d = 2^k
    return __dmul_rn(x, __longlong_as_double((1023ll - k) << 52));   // 2^-k
  }
  return __ddiv_rn(x, (double)d);
}

__device__ __forceinline__ float refine_level(float lo, float hi, int l, int G) {
  const double w = __dsub_rn((double)hi, (double)lo);
  const double t = div_g1(__dmul_rn(w, (double)l), G);
  return __double2float_rn(__dadd_rn((double)lo, t));
}

// The next interval: the best level +- one grid spacing, clipped to the domain.
__device__ __forceinline__ void refine_next(float center, float lo, float hi, float lo0,
                                            float hi0, int G, float& nlo, float& nhi) {
  const double sp = div_g1(__dsub_rn((double)hi, (double)lo), G);
  double a = __dsub_rn((double)center, sp), z = __dadd_rn((double)center, sp);
  if (a < (double)lo0) a = (double)lo0;
  if (z > (double)hi0) z = (double)hi0;
  nlo = __double2float_rn(a);
  nhi = __double2float_rn(z);
}

__device__ __forceinline__ void refine_layout(const RefineParams& p, const float* lo,
                                              const float* hi, float* lv) {
  const int l = threadIdx.x;
  if (l < p.G)
    for (int e = 0; e < 3; ++e) lv[e * kRefineMaxPoints + l] = refine_level(lo[e], hi[e], l, p.G);
}

__global__ void refine_init(RefineParams p) {
  RefineRoundDev* rounds = reinterpret_cast<RefineRoundDev*>(p.rounds);
  refine_layout(p, p.lo0, p.hi0, p.lv);
  if (threadIdx.x == 0) {
    for (int e = 0; e < 3; ++e) {
      rounds[0].lo[e] = p.lo0[e];
      rounds[0].hi[e] = p.hi0[e];
    }
    rounds[0].round = 0;
    *p.ticket = 0u;
  }
}

__global__ void refine_step(RefineParams p, int r) {
  RefineRoundDev* rounds = reinterpret_cast<RefineRoundDev*>(p.rounds);
  const float* cur = p.lv + (r & 1) * 3 * kRefineMaxPoints;
  const int G = p.G;
  long long b = rounds[r].best_index;
  if (b < 0 || b >= (long long)G * G * G) b = 0;  // only after a failed round
  const int lb[3] = {(int)(b / ((long long)G * G)), (int)((b / G) % G), (int)(b % G)};
  float nlo[3], nhi[3];
  for (int e = 0; e < 3; ++e)
    refine_next(cur[e * kRefineMaxPoints + lb[e]], rounds[r].lo[e], rounds[r].hi[e], p.lo0[e],
                p.hi0[e], G, nlo[e], nhi[e]);
  __syncthreads();  // every thread has read round r before round r + 1 is written
  if (threadIdx.x == 0) {
    for (int e = 0; e < 3; ++e) rounds[r].alloc[e] = cur[e * kRefineMaxPoints + lb[e]];
    *p.ticket = 0u;
  }
  if (r + 1 >= p.R) return;
  refine_layout(p, nlo, nhi, p.lv + ((r + 1) & 1) * 3 * kRefineMaxPoints);
  if (threadIdx.x == 0) {
    for (int e = 0; e < 3; ++e) {
      rounds[r + 1].lo[e] = nlo[e];
      rounds[r + 1].hi[e] = nhi[e];
    }
    rounds[r + 1].round = r + 1;
  }
}

// ------------------------------------------- coarse-to-fine, one cluster ---
// The whole refinement in one launch: a cluster of kRefineCluster CTAs (1,024
// threads each) evaluates a round's candidates, a warp per candidate as
// grid_batched does for grids of this size; each CTA publishes its top-2 in shared memory, every CTA
// reads all of them through distributed shared memory after a cluster
// barrier, and each lays out the next round itself (the same arithmetic, so
// the CTAs agree). A second cluster barrier keeps a round's top-2 readable
// until every CTA has read it. Results equal the launch-per-round form bit
// for bit; the per-round launches and their gaps disappear.

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

// Address of `local` (a shared variable) in the shared memory of cluster CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* local, uint32_t rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ TopTwo load_remote_top(const TopTwo* local, uint32_t rank) {
  const uint32_t a = cluster_addr(local, rank);
  TopTwo t;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(t.v1) : "r"(a) : "memory");
  asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(t.i1) : "r"(a + 8u) : "memory");
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(t.v2) : "r"(a + 16u) : "memory");
  return t;
}

__global__ void __cluster_dims__(kRefineCluster, 1, 1) __launch_bounds__(1024, 1)
    refine_fused(RefineFusedParams p) {
  extern __shared__ float sm[];              // positions [n_trials][6]
  __shared__ float lv[3][kRefineMaxPoints];  // this round's levels
  __shared__ float box[6];                   // this round's lo[3], hi[3]
  __shared__ TopTwo warp_best[32];
  __shared__ TopTwo cta_best;
  const uint32_t rank = cluster_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = 32 * kRefineCluster, gw = (int)rank * 32 + warp;
  const int G = p.G;
  RefineRoundDev* rounds = reinterpret_cast<RefineRoundDev*>(p.rounds);
  for (int i = tid; i < 6 * p.n_trials; i += blockDim.x) sm[i] = __ldg(p.pos + i);
  if (tid < 3) {
    box[tid] = p.lo0[tid];
    box[3 + tid] = p.hi0[tid];
  }
  __syncthreads();
  // one level per thread: thread e G + l computes level l of signal e
  if (tid < 3 * G) lv[tid / G][tid % G] = refine_level(box[tid / G], box[3 + tid / G], tid % G, G);
  __syncthreads();
  const long long n_cand = (long long)G * G * G;
  const double inv = 1.0 / (double)p.n_trials;
  for (int r = 0; r < p.R; ++r) {
    const uint32_t stream0 = (uint32_t)((long long)r * n_cand);
    TopTwo best = top_init();
    float kh = 0.f, kl = 0.f;
    long long kc = -1;
    int slot = 0;
    auto flush = [&]() {
      if (kc >= 0) best = top_merge(best, TopTwo{pair_mean(kh, kl, inv), kc, -DBL_MAX});
      kc = -1;
    };
    // candidates as grid_batched evaluates grids of this size (a round holds at
    // most 8,192 < kGridNarrowMin candidates: a whole warp per candidate)
    constexpr int kGridLanes = 32, kGridCandsPerWarp = 1;
    const int grp = lane / kGridLanes, gl = lane % kGridLanes;
    for (long long cb = (long long)gw * kGridCandsPerWarp; cb < n_cand;
         cb += (long long)W * kGridCandsPerWarp) {
      const long long c = cb + grp;
      float hi = 0.f, lo = 0.f;
      if (c < n_cand) {
        const uint32_t u = (uint32_t)c, q = u / (uint32_t)G;
        const int l2 = (int)(u - q * (uint32_t)G), l1 = (int)(q % (uint32_t)G),
                  l0 = (int)(q / (uint32_t)G);
        const float a0 = lv[0][l0], a1 = lv[1][l1], a2 = lv[2][l2];
        const float sd0 = 1.0f / (p.offset + a0), sd1 = 1.0f / (p.offset + a1),
                    sd2 = 1.0f / (p.offset + a2);
        const float cost = a0 * a0 + a1 * a1 + a2 * a2;
        for (int j = gl; j < p.n_trials; j += kGridLanes)
          two_sum_add(hi, lo, pp_outcome_at(p.rk, (uint32_t)j, stream0 + (uint32_t)c, 0u,
                                            sm + 6 * j, sd0, sd1, sd2, p.weight, cost));
      }
      group_pair_sum<kGridLanes>(hi, lo);
      const int g = lane - slot;
      const bool mine = g >= 0 && g < kGridCandsPerWarp;
      const int src = mine ? g * kGridLanes : 0;
      const float th = __shfl_sync(kFull, hi, src), tl = __shfl_sync(kFull, lo, src);
      if (mine && cb + g < n_cand) {
        kh = th;
        kl = tl;
        kc = cb + g;
      }
      slot += kGridCandsPerWarp;
      if (slot == 32) {
        flush();
        slot = 0;
      }
    }
    flush();
    best = top_warp(best);
    if (lane == 0) warp_best[warp] = best;
    __syncthreads();
    if (warp == 0) {
      const TopTwo t = top_warp(warp_best[lane]);
      if (lane == 0) cta_best = t;
    }
    cluster_sync_all();   // every CTA's top-2 is published
    if (warp == 0) {
      // lane q reads CTA q's top-2; the warp merges them
      TopTwo t = lane < kRefineCluster ? load_remote_top(&cta_best, (uint32_t)lane) : top_init();
      t = top_warp(t);
      long long b = t.i1;
      if (b < 0 || b >= n_cand) b = 0;
      const int lb[3] = {(int)(b / ((long long)G * G)), (int)((b / G) % G), (int)(b % G)};
      // lanes 0-2: the best level of signal `lane` and its next interval
      const int e = lane < 3 ? lane : 0;
      const float center = lv[e][lb[e]];
      float nlo = 0.f, nhi = 0.f;
      if (lane < 3) refine_next(center, box[e], box[3 + e], p.lo0[e], p.hi0[e], G, nlo, nhi);
      const float c0 = __shfl_sync(kFull, center, 0), c1 = __shfl_sync(kFull, center, 1),
                  c2 = __shfl_sync(kFull, center, 2);
      if (rank == 0 && lane == 0) {
        RefineRoundDev& o = rounds[r];
        o.alloc[0] = c0;
        o.alloc[1] = c1;
        o.alloc[2] = c2;
        for (int q = 0; q < 3; ++q) {
          o.lo[q] = box[q];
          o.hi[q] = box[3 + q];
        }
        o.round = r;
        o.best_index = t.i1;
        o.value = t.v1;
        o.gap = (t.v2 == -DBL_MAX) ? 0.0 : t.v1 - t.v2;
      }
      __syncwarp();
      if (lane < 3) {
        box[e] = nlo;
        box[3 + e] = nhi;
      }
    }
    cluster_sync_all();   // every CTA has read this round's top-2 (and this CTA's box is set)
    if (r + 1 < p.R) {
      if (tid < 3 * G)
        lv[tid / G][tid % G] = refine_level(box[tid / G], box[3 + tid / G], tid % G, G);
      __syncthreads();
    }
  }
}

size_t grid_smem(const GridParams& p) {
  return sizeof(float) * (6 * (size_t)p.n_trials + p.L[0] + p.L[1] + p.L[2]);
}

}  // namespace

int grid_blocks(int mode, long long n_cand, int n_trials, int lanes) {
  (void)n_trials;
  if (mode == 1) return (int)((n_cand + 255) / 256);
  int nb = 0;
  if (lanes == 8)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, grid_batched<8>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, grid_batched<32>, 256, 0);
  if (nb < 1) nb = 1;
  long long g = (long long)num_sms() * nb;
  const long long per_block = 8LL * (32 / lanes);
  const long long need = (n_cand + per_block - 1) / per_block;
  return (int)(g < need ? g : need);
}

cudaError_t launch_grid(const GridParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  const size_t smem = grid_smem(p);  // <= 6 * 1024 + 3 * 4096 floats (runtime limits)
  if (p.n_cand <= 0) return cudaSuccess;
  if (mode == 1) {
    cudaError_t ea = smem_limit((const void*)grid_plain, 96 * 1024);
    if (ea != cudaSuccess) return ea;
    const long long grid = (p.n_cand + 255) / 256;
    grid_plain<<<(unsigned)grid, 256, smem, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int ab = (int)((p.n_cand + 255) / 256);
    if (ab > 1024) ab = 1024;
    if (ab < 1) ab = 1;
    argmax_kernel<<<ab, 256, 0, s>>>(p.means, p.n_cand, p.cand0, p.partials, p.ticket,
                                     p.result);
    return cudaGetLastError();
  }
  const int block = (cfg.block == 128 || cfg.block == 256) ? cfg.block : 256;
  const int lanes = grid_lanes(p.L);
  int grid = cfg.grid > 0 ? cfg.grid : grid_blocks(0, p.n_cand, p.n_trials, lanes);
  if (grid > kMaxGridBlocks) grid = kMaxGridBlocks;  // one argmax partial per block
  const long long per_block = (long long)(block / 32) * (32 / lanes);
  const long long need = (p.n_cand + per_block - 1) / per_block;
  if (grid > need) grid = (int)need;
  cudaError_t ea = lanes == 8 ? smem_limit((const void*)grid_batched<8>, 96 * 1024)
                              : smem_limit((const void*)grid_batched<32>, 96 * 1024);
  if (ea != cudaSuccess) return ea;
  if (lanes == 8)
    grid_batched<8><<<grid, block, smem, s>>>(p);
  else
    grid_batched<32><<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_grid_batch(const GridBatchParams& p, cudaStream_t s) {
  const bool narrow = grid_lanes(p.L) == 8;
  int nb = 0;
  cudaError_t e = narrow
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, grid_batch<8>, 256, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, grid_batch<32>, 256, 0);
  if (e != cudaSuccess) return e;
  long long g = (long long)num_sms() * (nb > 0 ? nb : 1);
  const long long items = (long long)p.n_search * p.cpc;
  if (g > items) g = items;
  if (g < 1) return cudaSuccess;
  if (narrow)
    grid_batch<8><<<(unsigned)g, 256, 0, s>>>(p);
  else
    grid_batch<32><<<(unsigned)g, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_refine_fused(const RefineFusedParams& p, cudaStream_t s) {
  const size_t smem = sizeof(float) * 6 * (size_t)p.n_trials;
  refine_fused<<<kRefineCluster, 1024, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_refine_init(const RefineParams& p, cudaStream_t s) {
  refine_init<<<1, kRefineMaxPoints, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_refine_step(const RefineParams& p, int r, cudaStream_t s) {
  refine_step<<<1, kRefineMaxPoints, 0, s>>>(p, r);
  return cudaGetLastError();
}

cudaError_t launch_tie_reservoir(const double* v, long long n, long long base, uint64_t seed,
                                 void* result, cudaStream_t s) {
  tie_reservoir<<<1, 1024, 0, s>>>(v, n, base, (uint32_t)seed, (uint32_t)(seed >> 32), result);
  return cudaGetLastError();
}

cudaError_t launch_argmax(const double* v, long long n, TopTwo* partials, unsigned int* ticket,
                          void* result, cudaStream_t s) {
  long long g = (n + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  argmax_kernel<<<(unsigned)g, 256, 0, s>>>(v, n, 0, partials, ticket, result);
  return cudaGetLastError();
}

}  // namespace dg
