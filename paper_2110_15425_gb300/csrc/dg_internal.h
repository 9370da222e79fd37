// Internal interface between the host runtime (runtime.cpp) and the kernel
// translation units. Plain structs of device pointers and scalars; no torch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

// Launch shape chosen by the runtime (autotuned for the batched kernels).
struct LaunchCfg {
  int block = 256;   // threads per block
  int grid = 0;      // blocks; 0 = one per SM times occupancy
  int tpt = 1;       // threads per trial (LCA)
  int order = 0;     // LCA: 1 = hand trials out longest-expected-first
};

// ------------------------------------------------------------------ DDM ---
// The ten round keys of Philox4x32-10 for key (k0, k1): round r uses
// (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85). Passed in a kernel's parameters, a
// round's key words are constant-bank operands of its xor instructions.
struct PhiloxKeys {
  uint32_t k[20];
};
#ifdef __CUDACC__
#define DG_HD __host__ __device__
#else
#define DG_HD
#endif
DG_HD inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys r;
  for (int i = 0; i < 10; ++i) {
    r.k[2 * i] = k0 + (uint32_t)i * 0x9E3779B9u;
    r.k[2 * i + 1] = k1 + (uint32_t)i * 0xBB67AE85u;
  }
  return r;
}

// One job of a multi-job launch (DDM or LCA): the launch's trial list is the
// concatenation of its jobs' trials, job j holding list entries
// start .. start + n - 1; each job has its own inputs, outputs, seed and
// trial offset (the model's parameters are the launch's).
constexpr int kMaxMultiJobs = 256;   // table: 18 KB of kernel parameter space
struct MultiJob {
  long long start;
  long long n;
  const float* in;               // DDM: [2][n] (A row, z row); LCA: [n][N];
                                 // small network: [n_cond][input units]
  int8_t* choice;
  int32_t* step;
  float* xout;                   // may be null
  uint32_t trial0;
  uint32_t k0, k1;
  int32_t n_cond, cond_block;    // small network: condition of trial g is (g / cond_block) % n_cond
  uint32_t pad;
};
// The jobs of one multi-job launch, passed by value as a kernel parameter.
struct MultiJobTable {
  int n_jobs;
  MultiJob jobs[kMaxMultiJobs];
};

struct DdmParams {
  const float* A;      // [n] drift
  const float* z;      // [n] threshold
  int64_t n;
  uint32_t trial0;     // global id of local trial 0 (RNG counter)
  uint32_t k0, k1;     // Philox key
  float dt;            // Euler step (FP32 copy)
  float diffusion;     // sigma * sqrt(dt), rounded once from FP64
  float x0;
  int max_steps;
  int8_t* choice;
  int32_t* step;
  float* xout;         // may be null
  unsigned long long* cursor;  // batched form: global trial cursor (zeroed per launch)
  const unsigned int* perm;    // batched form: order in which trials are handed out (or null)
  PhiloxKeys rk;               // round keys of (k0, k1)
};
cudaError_t launch_ddm(const DdmParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s);
// Trials of several jobs of one DDM model in one persistent launch: p holds the
// model's parameters, p.n the total of the jobs' trials and p.cursor.
cudaError_t launch_ddm_multi(const DdmParams& p, const MultiJobTable& tab, cudaStream_t s);
int ddm_max_blocks_per_sm(int block);

// ------------------------------------------------------------------ LCA ---
struct LcaParams {
  const float* I;      // [n][N]
  int64_t n;
  uint32_t trial0;
  int N;
  uint32_t k0, k1;
  float dt, diffusion, leak, inhibition, threshold;
  int max_steps;
  int rectify, two_sided;
  int8_t* choice;
  int32_t* step;
  float* xout;         // [n][N], may be null
  unsigned long long* cursor;
  const unsigned int* perm;    // batched form: hand-out order (or null)
  PhiloxKeys rk;                 // round keys of (k0, k1)
  int chunk;                     // compacting form: steps between compactions
  int tail_max;                  // compacting form: at most this many trials left -> a warp each
};
cudaError_t launch_lca(const LcaParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s);
// Trials of several jobs of one LCA model in one persistent launch (a lane per
// trial; p holds the model's parameters, p.n the total and p.cursor).
cudaError_t launch_lca_multi(const LcaParams& p, const MultiJobTable& tab, cudaStream_t s);
bool lca_tpt_supported(int N, int tpt);
int lca_max_blocks_per_sm(int N, int tpt, int block);

// ---------------------------------------------------- small logistic network ---
constexpr int kNetMaxUnits = 32;     // logistic units
constexpr int kNetMaxInputs = 64;    // input units
constexpr int kNetMaxInDegree = 32;  // incoming edges from logistic units, per unit
constexpr int kNetMaxDdm = 8;        // DDM nodes on the stop layer (Extended Stroop)
constexpr int kNetMaxStop = 16;      // stop-layer units

// Static layout of a small network (Sec. 3.3): logistic units numbered in
// mechanism order; unit u's incoming edges from logistic units are the dense
// row src[u][0..D), w[u][0..D) (in projection order, padded with weight 0);
// the input part of each net input is a [U][n_in] matrix applied once per trial.
struct NetLayout {
  int U;                         // logistic units
  int n_in;                      // input units
  int D;                         // incoming-edge row length
  int stop_off, stop_size;       // stop layer among logistic units
  float rate, noise;
  float stop_threshold;
  int max_steps;
  float gain[kNetMaxUnits];
  float bias[kNetMaxUnits];
  float w[kNetMaxUnits][kNetMaxInDegree];
  int8_t src[kNetMaxUnits][kNetMaxInDegree];
  // DDM nodes driven by the stop layer once the network stops (0 = none):
  // drift_q = ddm_bias[q] + sum_i ddm_w[q][i] y_i, then x += drift dt + diffusion eps
  int n_ddm;
  float ddm_w[kNetMaxDdm][kNetMaxStop];
  float ddm_bias[kNetMaxDdm];
  float ddm_dt[kNetMaxDdm];
  float ddm_diffusion[kNetMaxDdm];   // sigma sqrt(dt)
  float ddm_z[kNetMaxDdm];           // bound
  int ddm_max[kNetMaxDdm];           // steps
};

struct NetParams {
  const NetLayout* layout;       // device copy
  const float* w_in;             // device [U][n_in]
  const float* cond;             // device [n_cond][n_in]
  int n_cond, cond_block;
  int64_t n;
  uint32_t trial0;
  uint32_t k0, k1;
  int U, n_in, stop_size;        // host copies for launch sizing
  int n_ddm;                     // host copy
  int state_size;                // floats per trial in yout: stop_size (+ 3 per DDM node)
  int8_t* choice;
  int32_t* step;
  float* yout;                   // [n][state_size], may be null
  unsigned long long* cursor;
  PhiloxKeys rk;                 // round keys of (k0, k1)
};
cudaError_t launch_net(const NetParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s);

// One lane per trial for networks of at most kLaneMaxU logistic units (and
// their DDM nodes, run after the network in the same lane): the incoming-edge
// table as a dense matrix (W[u][v] the weight of
// the edge from unit v into unit u, 0 where there is none), passed by value.
constexpr int kLaneMaxU = 8;
struct NetDense {
  float W[kLaneMaxU][kLaneMaxU];
  float gain[kLaneMaxU], bias[kLaneMaxU];
  float rate, noise, thr;
  int stop_off, stop_size, max_steps;
  // DDM nodes on the stop layer (Extended Stroop; n_ddm = 0: none), as in NetLayout
  int n_ddm;
  float ddm_w[kNetMaxDdm][kNetMaxStop];
  float ddm_bias[kNetMaxDdm], ddm_dt[kNetMaxDdm], ddm_diffusion[kNetMaxDdm], ddm_z[kNetMaxDdm];
  int ddm_max[kNetMaxDdm];
};
cudaError_t launch_net_lane(const NetParams& p, const NetDense& q, cudaStream_t s);
// Trials of several jobs of one such network in one launch (p: the model's
// part, p.n the total of the jobs' trials and p.cursor).
cudaError_t launch_net_lane_multi(const NetParams& p, const NetDense& q, const MultiJobTable& tab,
                                  cudaStream_t s);

// --------------------------------------------------- wide network (tensor cores) ---
struct WideParams {
  const float* w_in;             // [H][S + T] FP32: stimulus and task weights side by side
  const uint16_t* w_resp_bf16;   // shared-memory image of the MMA B operand: [16][2H]
                                 // bfloat16 (W | W) in the K-major canonical layout
  const float* w_resp_f32;       // [16][H] FP32 copy of the same bf16 values (plain kernel)
  const float* cond;             // [n_cond][S + T] one-hot rows
  int n_cond, cond_block;
  int S, T, H, R;
  float bias_h, bias_r, gain_h, gain_r, rate, noise, stop_threshold;
  int max_steps;
  int64_t n;
  uint32_t trial0;
  uint32_t k0, k1;
  int8_t* choice;
  int32_t* step;
  float* yout;                   // [n][R], may be null
  unsigned long long* cursor;
  int* status;                   // device status word (bounded mbarrier waits)
  PhiloxKeys rk;                 // round keys of (k0, k1)
  float* net_table;              // scratch [n_cond][H]: hidden net input per condition
};
cudaError_t launch_wide(const WideParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s);
size_t wide_smem_bytes(int H, int nin, bool tc);
void wide_b_image(const uint16_t* w_bf16, int H, uint16_t* img);

// ------------------------------------------------------- predator-prey grid ---
struct TopTwo {                  // running argmax with lowest-index ties
  double v1;
  long long i1;
  double v2;
};

constexpr int kMaxGridBlocks = 4096;  // size of the per-block argmax partials scratch
// Batched grid search: lanes per candidate (its trials spread over them).
// Grids of at least kGridNarrowMin candidates take eight lanes per candidate
// (four candidates per warp: the per-candidate work is shared by fewer lanes);
// smaller grids a whole warp, so that a round of a few hundred candidates
// still spreads over many warps. The choice depends on the whole grid's size
// only, so a candidate's mean has the same bits whatever range a call
// evaluates and whatever the launch shape.
constexpr long long kGridNarrowMin = 16384;
inline int grid_lanes(const int (&L)[3]) {
  return (long long)L[0] * L[1] * L[2] >= kGridNarrowMin ? 8 : 32;
}

struct GridParams {
  const float* lv[3];
  int L[3];
  const float* pos;              // [n_trials][6]
  int n_trials;
  uint32_t k0, k1;
  float offset, weight;
  long long cand0;               // global index of local candidate 0
  long long n_cand;              // candidates evaluated by this launch
  uint32_t stream0;              // noise stream of candidate c is stream0 + c
  double* means;                 // [n_cand] local, may be null
  TopTwo* partials;              // scratch, one per block
  unsigned int* ticket;          // scratch, zeroed per launch
  void* result;                  // dg_grid_result*
  PhiloxKeys rk;                 // round keys of (k0, k1)
};
cudaError_t launch_grid(const GridParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s);
int grid_blocks(int mode, long long n_cand, int n_trials, int lanes);

cudaError_t launch_argmax(const double* v, long long n, TopTwo* partials, unsigned int* ticket,
                          void* result, cudaStream_t s);

// A batch of whole-grid searches of one predator-prey model in one launch: the
// searches share the grid shape (levels per signal, trials per candidate) and
// each has its own level values, positions, seed and outputs.
constexpr int kMaxGridBatch = 256;
constexpr int kGridChunk = 128;    // candidates per work item
struct GridBatchItem {
  const float* lv[3];
  const float* pos;                // [n_trials][6]
  void* result;                    // dg_grid_result*
  double* means;                   // [n_cand] or null
  uint32_t k0, k1;                 // Philox key of the search's seed
};
struct GridBatchParams {
  int L[3];
  int n_trials;
  float offset, weight;
  long long n_cand;
  int cpc;                         // chunks per search
  int n_search;
  unsigned long long* cursor;      // scratch, zeroed per launch
  unsigned int* ticket;            // scratch [n_search], zeroed per launch
  TopTwo* partials;                // scratch [n_search][cpc]
  GridBatchItem items[kMaxGridBatch];
};
cudaError_t launch_grid_batch(const GridBatchParams& p, cudaStream_t s);
// --------------------------------------------- predator-prey episodes ---
constexpr int kEpisodeChunk = 64;   // candidates per work item (8 warps x 8)
struct EpisodeParams {
  const float* lv[3];
  int L[3];
  long long n_cand;
  int cpe;                       // work items (candidate chunks) per episode
  int n_trials;
  uint32_t k0, k1;
  float offset, weight;          // FP32 copies for the candidate simulations
  double offset_d, weight_d;     // the model's values, for the FP64 moves
  double speed[3];               // player, predator, prey
  double radius;
  int E, T;                      // episodes, maximum steps
  uint32_t e0;                   // global index of episode 0
  int t;                         // the step a launch performs
  const float* start;            // [E][6]
  float* state;                  // [E][6] positions at the start of the step
  int* active;                   // [3][E] active episode lists, rotating by step
  int* count;                    // [3] list lengths
  unsigned long long* cursor;    // [3] next work item of the step
  unsigned int* ticket;          // [E] finished work items of the step
  TopTwo* partials;              // [E][cpe]
  int8_t* outcome;               // [E]
  int32_t* steps;                // [E]
  float* final_pos;              // [E][6] or null
  int32_t* traj_best;            // [E][T] or null
  double* traj_value;            // [E][T] or null
  float* traj_pos;               // [E][T][6] or null
  PhiloxKeys rk;                 // round keys of (k0, k1)
};
cudaError_t launch_episode_init(const EpisodeParams& p, cudaStream_t s);
cudaError_t launch_episode_step(const EpisodeParams& p, cudaStream_t s);

// ------------------------------------------------- coarse-to-fine grid ---
constexpr int kRefineMaxPoints = 64;
struct RefineParams {
  float lo0[3], hi0[3];          // domain of each signal
  int G;                         // points per signal per round
  int R;                         // rounds
  float* lv;                     // scratch [2][3][kRefineMaxPoints]: levels, double-buffered
  void* rounds;                  // dg_refine_round[R]
  unsigned int* ticket;          // the grid launch's argmax ticket, reset for the next round
};
// The whole refinement in one launch of one thread-block cluster.
constexpr int kRefineCluster = 8;
struct RefineFusedParams {
  float lo0[3], hi0[3];
  int G, R, n_trials;
  const float* pos;              // [n_trials][6]
  PhiloxKeys rk;
  float offset, weight;
  void* rounds;                  // dg_refine_round[R]
};
cudaError_t launch_refine_fused(const RefineFusedParams& p, cudaStream_t s);
// Levels and box of round 0.
cudaError_t launch_refine_init(const RefineParams& p, cudaStream_t s);
// After round r's grid launch: record the best allocation and lay out round r + 1.
cudaError_t launch_refine_step(const RefineParams& p, int r, cudaStream_t s);

// After an argmax into `result` over v[0..n) (global indices base..): replace
// the lowest tied index by the reservoir-sampled one when the maximum is tied.
cudaError_t launch_tie_reservoir(const double* v, long long n, long long base, uint64_t seed,
                                 void* result, cudaStream_t s);

// ------------------------------------------- longest-expected-first order ---
constexpr int kSchedBuckets = 1024;

struct SchedParams {
  int kind;                      // 0 DDM, 1 LCA
  const float* a;                // DDM: A[n]; LCA: I[n][N]
  const float* b;                // DDM: z[n]
  int N;
  long long n;
  float dt, sigma2, leak, inhibition, threshold;
  int max_steps;
  unsigned int* hist;            // [kSchedBuckets] scratch
  unsigned int* cursor;          // [kSchedBuckets] scratch
  unsigned int* perm;            // [n] output
  unsigned short* bucket;        // [n] scratch: each trial's bucket
};
cudaError_t launch_sched(const SchedParams& s, cudaStream_t st);

// ------------------------------------------------------------ RNG replay ---
cudaError_t launch_philox_words(uint64_t seed, uint32_t trial, uint32_t cand, uint32_t purpose,
                                uint32_t block0, int64_t nblocks, uint32_t* out, cudaStream_t s);
cudaError_t launch_normals(uint64_t seed, uint32_t trial, uint32_t cand, uint64_t d0, int64_t n,
                           float* out, cudaStream_t s);

cudaError_t launch_wait_timeout(long long limit_cycles, int* status, cudaStream_t s);
// The grid search's per-candidate reduction on given values (lanes 8 or 32).
cudaError_t launch_pair_sum(const float* x, long long n_groups, int per, int lanes,
                            double* means, cudaStream_t s);

// Multiprocessors of the current device (looked up once per device).
int num_sms();

// Raise the dynamic shared-memory limit of kernel `fn` to at least `bytes` on
// the current device. The attribute is per device, so it is set once per
// (kernel, device) pair and again only when a larger limit is asked for;
// thread-safe. Returns the CUDA error of the attribute call, if any.
cudaError_t smem_limit(const void* fn, int bytes);

}  // namespace dg
