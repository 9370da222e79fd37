// Host runtime of the C ABI in include/distill_gpu.h: compose-time validation
// and static layout (Sec. 2.2 sanitization, Sec. 3.3 static structures),
// launch dispatch, per-stream scratch, the launch-shape autotuner, CUDA-graph
// batches and the continuous-batching serving loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "distill_gpu.h"
#include "dg_device.cuh"
#include "dg_internal.h"

// ----------------------------------------------------------------- errors ---

namespace {

thread_local std::string g_err = "no error";

dg_status fail(dg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define DG_CUDA(x)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) return fail(DG_E_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ModelKind { K_DDM = 0, K_LCA = 1, K_NET = 2, K_WIDE = 3, K_PP = 4 };

// Per-stream scratch: trial cursor, argmax ticket, device status word, the
// histogram and bucket cursors of the trial-order sort, per-block argmax
// partials; plus growable buffers for the trial order and for the plain grid
// search's means.
constexpr size_t kMaxPartials = dg::kMaxGridBlocks;
constexpr size_t kSortOff = 256;
constexpr size_t kScratchHead = kSortOff + 2 * dg::kSchedBuckets * sizeof(unsigned int) + 256;
constexpr size_t kRefineOff = kScratchHead + kMaxPartials * sizeof(dg::TopTwo);
constexpr size_t kScratchBytes = kRefineOff + 2 * 3 * dg::kRefineMaxPoints * sizeof(float);

struct Scratch {
  unsigned char* base = nullptr;
  double* means = nullptr;
  size_t means_cap = 0;
  unsigned int* perm = nullptr;
  size_t perm_cap = 0;
  unsigned char* ext = nullptr;  // episodes: state, lists, tickets, partials
  size_t ext_cap = 0;
  unsigned char* gb = nullptr;   // batched grid searches: cursor, tickets, partials
  size_t gb_cap = 0;
  float* net = nullptr;          // wide network: hidden net input per condition
  size_t net_cap = 0;
  unsigned long long* cursor() { return reinterpret_cast<unsigned long long*>(base); }
  unsigned int* ticket() { return reinterpret_cast<unsigned int*>(base + 8); }
  int* status() { return reinterpret_cast<int*>(base + 16); }
  unsigned int* hist() { return reinterpret_cast<unsigned int*>(base + kSortOff); }
  unsigned int* bucket_cursor() { return hist() + dg::kSchedBuckets; }
  dg::TopTwo* partials() { return reinterpret_cast<dg::TopTwo*>(base + kScratchHead); }
  float* refine_levels() { return reinterpret_cast<float*>(base + kRefineOff); }
};

struct Server;

}  // namespace

struct dg_ctx {
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::unordered_map<cudaStream_t, Scratch> scratch;
  std::map<std::string, dg::LaunchCfg> tuned;
  std::string tune_file;
  bool autotune = true;
  // launches that ran a default shape because their key had no tuned shape
  // and tuning was not allowed there (serving thread, graph capture)
  std::atomic<int64_t> untuned{0};
  std::unique_ptr<Server> server;
  std::mutex server_mu;
};

struct dg_model {
  dg_ctx* ctx = nullptr;
  int kind = 0;
  int max_steps = 1;
  // DDM
  float dt = 0.f, diffusion = 0.f, x0 = 0.f, sigma = 0.f;
  // LCA
  int N = 0;
  float leak = 0.f, inhibition = 0.f, threshold = 0.f;
  int rectify = 1, two_sided = 0;
  // small network
  dg::NetLayout layout{};
  dg::NetLayout* d_layout = nullptr;
  float* d_w_in = nullptr;
  // wide network
  int S = 0, T = 0, H = 0, R = 0;
  float bias_h = 0, bias_r = 0, gain_h = 1, gain_r = 1, rate = 0, noise = 0, stop_thr = 0;
  float* d_w_hid = nullptr;  // wide: [H][S + T]
  uint16_t* d_w_resp_bf16 = nullptr;
  float* d_w_resp_f32 = nullptr;
  // predator-prey
  float offset = 0.f, weight = 0.f;
  double offset_d = 0.0, weight_d = 0.0;  // as given, for the FP64 episode moves
  int state_size = 0;
  int n_inputs = 0;  // TRANSFER: input units per condition row
  std::vector<std::vector<float>> proj_w;  // FP32 weights of each projection (empty: structural)
};

namespace {

// ------------------------------------------------------------ scratch ---

dg_status get_scratch(dg_ctx* ctx, cudaStream_t s, Scratch** out) {
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->scratch.find(s);
  if (it == ctx->scratch.end()) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return fail(DG_E_STATE,
                  "first use of a stream must not be inside stream capture (scratch allocation)");
    Scratch sc;
    DG_CUDA(cudaMalloc(&sc.base, kScratchBytes));
    // zeroed on the stream itself: a plain cudaMemset runs on the legacy
    // stream, which does not order against non-blocking streams
    DG_CUDA(cudaMemsetAsync(sc.base, 0, kScratchBytes, s));
    it = ctx->scratch.emplace(s, sc).first;
  }
  *out = &it->second;
  return DG_OK;
}

dg_status scratch_means(dg_ctx* ctx, Scratch* sc, size_t n, cudaStream_t s) {
  if (sc->means_cap >= n) return DG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(DG_E_STATE, "plain grid search needs a means buffer; run once before capture");
  std::lock_guard<std::mutex> g(ctx->mu);
  DG_CUDA(cudaStreamSynchronize(s));
  if (sc->means) cudaFree(sc->means);
  sc->means = nullptr;
  DG_CUDA(cudaMalloc(&sc->means, n * sizeof(double)));
  sc->means_cap = n;
  return DG_OK;
}

dg_status scratch_ext(dg_ctx* ctx, Scratch* sc, size_t n, cudaStream_t s) {
  if (sc->ext_cap >= n) return DG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(DG_E_STATE, "episodes need scratch of this size; run once before capture");
  std::lock_guard<std::mutex> g(ctx->mu);
  DG_CUDA(cudaStreamSynchronize(s));
  if (sc->ext) cudaFree(sc->ext);
  sc->ext = nullptr;
  DG_CUDA(cudaMalloc(&sc->ext, n));
  sc->ext_cap = n;
  return DG_OK;
}

dg_status scratch_gb(dg_ctx* ctx, Scratch* sc, size_t bytes, cudaStream_t s) {
  if (sc->gb_cap >= bytes) return DG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(DG_E_STATE, "grid search batch: scratch must grow; run this size once before capture");
  std::lock_guard<std::mutex> g(ctx->mu);
  DG_CUDA(cudaStreamSynchronize(s));
  if (sc->gb) cudaFree(sc->gb);
  sc->gb = nullptr;
  DG_CUDA(cudaMalloc(&sc->gb, bytes));
  sc->gb_cap = bytes;
  return DG_OK;
}

dg_status scratch_net(dg_ctx* ctx, Scratch* sc, size_t n, cudaStream_t s) {
  if (sc->net_cap >= n) return DG_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(DG_E_STATE, "wide network: per-condition table must grow; run once before capture");
  std::lock_guard<std::mutex> g(ctx->mu);
  DG_CUDA(cudaStreamSynchronize(s));
  if (sc->net) cudaFree(sc->net);
  sc->net = nullptr;
  DG_CUDA(cudaMalloc(&sc->net, n * sizeof(float)));
  sc->net_cap = n;
  return DG_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

dg_status scratch_perm(dg_ctx* ctx, Scratch* sc, size_t n, cudaStream_t s) {
  if (sc->perm_cap >= n) return DG_OK;
  if (capturing(s))
    return fail(DG_E_STATE, "trial-order buffer must grow; run this size once before capture");
  std::lock_guard<std::mutex> g(ctx->mu);
  DG_CUDA(cudaStreamSynchronize(s));
  if (sc->perm) cudaFree(sc->perm);
  sc->perm = nullptr;
  // permutation (4 B per trial) followed by each trial's bucket (2 B per trial)
  DG_CUDA(cudaMalloc(&sc->perm, n * (sizeof(unsigned int) + sizeof(unsigned short))));
  sc->perm_cap = n;
  return DG_OK;
}

// Longest-expected-first hand-out order (DG_LPT=0 turns it off). Small jobs
// skip it: their launch is not long enough for the order to matter.
bool lpt_enabled(long long n) {
  static const int on = [] {
    const char* e = getenv("DG_LPT");
    return e ? atoi(e) : 1;
  }();
  return on && n >= 4096;
}

// Set on the serving thread: never time launch shapes there (tuning
// synchronizes); use tuned shapes when known, defaults otherwise.
thread_local bool t_no_tune = false;

// ---------------------------------------------------------- autotuner ---

void load_tune_file(dg_ctx* ctx) {
  if (ctx->tune_file.empty()) return;
  FILE* f = fopen(ctx->tune_file.c_str(), "r");
  if (!f) return;
  char line[512], key[256];
  while (fgets(line, sizeof line, f)) {
    int b, g, t, o = 0;
    if (sscanf(line, "%255s %d %d %d %d", key, &b, &g, &t, &o) < 4) continue;
    dg::LaunchCfg c;
    c.block = b;
    c.grid = g;
    c.tpt = t;
    c.order = o;
    ctx->tuned[key] = c;
  }
  fclose(f);
}

void save_tune_file(dg_ctx* ctx) {
  if (ctx->tune_file.empty()) return;
  FILE* f = fopen(ctx->tune_file.c_str(), "w");
  if (!f) return;
  for (auto& kv : ctx->tuned)
    fprintf(f, "%s %d %d %d %d\n", kv.first.c_str(), kv.second.block, kv.second.grid,
            kv.second.tpt, kv.second.order);
  fclose(f);
}

int log2_bucket(long long n) {
  int b = 0;
  while ((1ll << b) < n && b < 62) ++b;
  return b;
}

// Launch `fn(cfg)` for each candidate shape, time each (best of 2) with
// events on the stream, keep the fastest (a later candidate only when it is
// more than 2 % faster). All candidates compute identical
// outputs (results depend only on inputs and seed), so the outputs left by
// the last run are the job's outputs.
template <class F>
dg_status autotune(dg_ctx* ctx, const std::string& key, const std::vector<dg::LaunchCfg>& cands,
                   cudaStream_t s, F&& fn, dg::LaunchCfg* chosen, bool* ran) {
  *ran = false;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
      *chosen = it->second;
      return DG_OK;
    }
  }
  if (!ctx->autotune || t_no_tune || capturing(s) || cands.size() == 1) {
    if (ctx->autotune && cands.size() > 1) ctx->untuned.fetch_add(1);
    *chosen = cands.front();
    return DG_OK;
  }
  cudaEvent_t a, b;
  DG_CUDA(cudaEventCreate(&a));
  DG_CUDA(cudaEventCreate(&b));
  float best_ms = 1e30f;
  dg::LaunchCfg best = cands.front();
  for (const auto& c : cands) {
    float ms_best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(a, s);
      dg_status st = fn(c);
      if (st != DG_OK) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return st;
      }
      cudaEventRecord(b, s);
      if (cudaEventSynchronize(b) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      ms_best = std::min(ms_best, ms);
    }
    // a later candidate must be clearly faster: shapes that time within noise
    // of each other alone keep the default (the first listed), so that the
    // choice does not flip from run to run
    if (ms_best < best_ms * 0.98f) {
      best_ms = ms_best;
      best = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  // leave the job's outputs from the chosen shape
  dg_status st = fn(best);
  if (st != DG_OK) return st;
  *ran = true;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->tuned[key] = best;
    save_tune_file(ctx);
  }
  *chosen = best;
  return DG_OK;
}

// Run a batched launch with the tuned shape for `key` (tuning it first when
// it is unknown and the stream is not being captured).
template <class F>
dg_status run_tuned(dg_ctx* ctx, const std::string& key, const std::vector<dg::LaunchCfg>& cands,
                    cudaStream_t s, F&& go) {
  dg::LaunchCfg c;
  bool ran = false;
  dg_status st = autotune(ctx, key, cands, s, go, &c, &ran);
  if (st != DG_OK) return st;
  return ran ? DG_OK : go(c);
}

// Launch shapes: fewer resident trials per SM make each trial advance
// faster (the longest trials set a persistent launch's end) at the price of
// less latency hiding; the tuner measures where the balance lies.
std::vector<dg::LaunchCfg> ddm_candidates() {
  std::vector<dg::LaunchCfg> v;
  const int occ = dg::ddm_max_blocks_per_sm(256);
  for (int per_sm : {occ, 6, 5, 4, 3, 2}) {
    if (per_sm > occ || per_sm < 1) continue;
    if (!v.empty() && per_sm == occ) continue;
    dg::LaunchCfg c;
    c.block = 256;
    c.grid = dg::num_sms() * per_sm;
    v.push_back(c);
  }
  return v;
}

// DG_LCA_TPT=<1|2|4> restricts the threads-per-trial layouts the tuner may
// pick (used to exercise every layout).
int forced_tpt() {
  const char* e = getenv("DG_LCA_TPT");
  return e ? atoi(e) : 0;
}

// Hand-out order: longest-expected-first pays when lanes take new trials
// (the long ones start first); when every trial has a lane from the start it
// only gathers the longest trials into the same few blocks, which then run
// them side by side to the end. Each shape is offered in both orders, the one
// expected to win first (the default when the tuner does not run).
// DG_LCA_ORDER=<0|1> restricts the hand-out order likewise (0 as given, 1
// longest-expected-first).
int forced_order() {
  const char* e = getenv("DG_LCA_ORDER");
  return e ? atoi(e) : -1;
}

std::vector<dg::LaunchCfg> lca_candidates(int N, long long n, bool lpt) {
  std::vector<dg::LaunchCfg> v;
  const int only = forced_tpt(), order = forced_order();
  // tpt 0: one lane per trial with block-level compaction of running trials
  for (int tpt : {0, 1, 2, 4}) {
    if (!dg::lca_tpt_supported(N, tpt) || (only > 0 && tpt != only) || (only < 0 && tpt != 0))
      continue;
    const int occ = std::max(1, dg::lca_max_blocks_per_sm(N, tpt, 256));
    for (int div : {1, 2, 4}) {
      if (div > 1 && occ / div < 1) continue;
      dg::LaunchCfg c;
      c.block = 256;
      c.tpt = tpt;
      c.grid = dg::num_sms() * std::max(1, occ / div);
      const long long lanes = (long long)c.grid * c.block / std::max(1, tpt);
      c.order = lpt && n > lanes ? 1 : 0;
      for (int k = 0; k < (lpt ? 2 : 1); ++k, c.order ^= 1)
        if (order < 0 || !lpt || c.order == order) v.push_back(c);
    }
  }
  return v;
}

std::vector<dg::LaunchCfg> grid_candidates(long long n_cand, int lanes) {
  std::vector<dg::LaunchCfg> v;
  const int full = dg::grid_blocks(0, n_cand, 64, lanes);
  for (int per_warp : {0, 2, 3, 4}) {
    dg::LaunchCfg c;
    c.block = 256;
    if (per_warp == 0) {
      c.grid = full;
    } else {
      const long long per_block = 8LL * per_warp * (32 / lanes);
      long long g = (n_cand + per_block - 1) / per_block;
      if (g > (long long)kMaxPartials) continue;
      c.grid = (int)g;
    }
    v.push_back(c);
  }
  return v;
}

// ---------------------------------------------------------- run paths ---

// Small networks (with or without DDM nodes) run one lane per trial unless
// DG_NET_LANE=0 (then a lane group per trial).
bool net_lane_enabled() {
  const char* e = getenv("DG_NET_LANE");
  return !e || atoi(e) != 0;
}

// A small network that the one-lane form runs (at most kLaneMaxU logistic
// units, no DDM nodes), and its dense edge matrix.
bool net_lane_model(const dg_model* m) {
  return m->kind == K_NET && m->layout.n_ddm == 0 && m->layout.U <= dg::kLaneMaxU;
}

dg::NetDense net_dense(const dg::NetLayout& L) {
  dg::NetDense q{};
  for (int u = 0; u < L.U; ++u) {
    for (int d = 0; d < L.D; ++d)
      if (L.w[u][d] != 0.f) q.W[u][L.src[u][d]] = L.w[u][d];
    q.gain[u] = L.gain[u];
    q.bias[u] = L.bias[u];
  }
  q.rate = L.rate;
  q.noise = L.noise;
  q.thr = L.stop_threshold;
  q.stop_off = L.stop_off;
  q.stop_size = L.stop_size;
  q.max_steps = L.max_steps;
  q.n_ddm = L.n_ddm;
  for (int n = 0; n < L.n_ddm; ++n) {
    for (int i = 0; i < L.stop_size; ++i) q.ddm_w[n][i] = L.ddm_w[n][i];
    q.ddm_bias[n] = L.ddm_bias[n];
    q.ddm_dt[n] = L.ddm_dt[n];
    q.ddm_diffusion[n] = L.ddm_diffusion[n];
    q.ddm_z[n] = L.ddm_z[n];
    q.ddm_max[n] = L.ddm_max[n];
  }
  return q;
}

// The model's part of a DDM or LCA launch (the per-call part is set by the caller).
dg::DdmParams ddm_model_params(const dg_model* m) {
  dg::DdmParams p{};
  p.dt = m->dt;
  p.diffusion = m->diffusion;
  p.x0 = m->x0;
  p.max_steps = m->max_steps;
  return p;
}

dg::LcaParams lca_model_params(const dg_model* m) {
  dg::LcaParams p{};
  p.N = m->N;
  p.dt = m->dt;
  p.diffusion = m->diffusion;
  p.leak = m->leak;
  p.inhibition = m->inhibition;
  p.threshold = m->threshold;
  p.max_steps = m->max_steps;
  p.rectify = m->rectify;
  p.two_sided = m->two_sided;
  const char* e = getenv("DG_LCA_CHUNK");   // steps between compactions
  p.chunk = e && atoi(e) > 0 ? atoi(e) : 32;
  const char* tm = getenv("DG_LCA_TAIL");   // trials left in a block before a warp each
  p.tail_max = tm ? std::max(0, std::min(8, atoi(tm))) : 8;
  return p;
}

dg_status run_device(dg_model* m, const dg_run_desc* d, int8_t* choice, int32_t* step,
                     float* fs, cudaStream_t s) {
  if (d->n_trials == 0) return DG_OK;
  Scratch* sc = nullptr;
  dg_status st = get_scratch(m->ctx, s, &sc);
  if (st != DG_OK) return st;
  const uint32_t k0 = (uint32_t)d->seed, k1 = (uint32_t)(d->seed >> 32);
  const int mode = d->mode;
  const std::string bucket = std::to_string(log2_bucket(d->n_trials));

  if (m->kind == K_DDM) {
    dg::DdmParams p = ddm_model_params(m);
    p.A = d->trial_params;
    p.z = d->trial_params + d->n_trials;
    p.n = d->n_trials;
    p.trial0 = (uint32_t)d->trial_offset;
    p.k0 = k0;
    p.k1 = k1;
    p.rk = dg::philox_keys(k0, k1);
    p.choice = choice;
    p.step = step;
    p.xout = fs;
    p.cursor = sc->cursor();
    auto go = [&](const dg::LaunchCfg& c) -> dg_status {
      if (mode == DG_MODE_BATCHED) DG_CUDA(cudaMemsetAsync(sc->cursor(), 0, 8, s));
      DG_CUDA(dg::launch_ddm(p, mode, c, s));
      return DG_OK;
    };
    if (mode == DG_MODE_PLAIN) return go(dg::LaunchCfg{});
    if (lpt_enabled(d->n_trials)) {
      if ((st = scratch_perm(m->ctx, sc, (size_t)d->n_trials, s)) != DG_OK) return st;
      dg::SchedParams sp{};
      sp.kind = 0;
      sp.a = p.A;
      sp.b = p.z;
      sp.n = p.n;
      sp.dt = m->dt;
      sp.sigma2 = m->sigma * m->sigma;
      sp.max_steps = m->max_steps;
      sp.hist = sc->hist();
      sp.cursor = sc->bucket_cursor();
      sp.perm = sc->perm;
      sp.bucket = reinterpret_cast<unsigned short*>(sc->perm + sc->perm_cap);
      DG_CUDA(dg::launch_sched(sp, s));
      p.perm = sc->perm;
    }
    return run_tuned(m->ctx, "ddm/" + bucket, ddm_candidates(), s, go);
  }
  if (m->kind == K_LCA) {
    dg::LcaParams p = lca_model_params(m);
    p.I = d->trial_params;
    p.n = d->n_trials;
    p.trial0 = (uint32_t)d->trial_offset;
    p.k0 = k0;
    p.k1 = k1;
    p.rk = dg::philox_keys(k0, k1);
    p.choice = choice;
    p.step = step;
    p.xout = fs;
    p.cursor = sc->cursor();
    const bool lpt = mode == DG_MODE_BATCHED && lpt_enabled(d->n_trials) && !m->two_sided;
    if (lpt && (st = scratch_perm(m->ctx, sc, (size_t)d->n_trials, s)) != DG_OK) return st;
    auto go = [&](const dg::LaunchCfg& c) -> dg_status {
      p.perm = nullptr;
      if (lpt && c.order == 1) {
        dg::SchedParams sp{};
        sp.kind = 1;
        sp.a = p.I;
        sp.N = m->N;
        sp.n = p.n;
        sp.dt = m->dt;
        sp.leak = m->leak;
        sp.inhibition = m->inhibition;
        sp.threshold = m->threshold;
        sp.max_steps = m->max_steps;
        sp.hist = sc->hist();
        sp.cursor = sc->bucket_cursor();
        sp.perm = sc->perm;
        sp.bucket = reinterpret_cast<unsigned short*>(sc->perm + sc->perm_cap);
        DG_CUDA(dg::launch_sched(sp, s));
        p.perm = sc->perm;
      }
      if (mode == DG_MODE_BATCHED) DG_CUDA(cudaMemsetAsync(sc->cursor(), 0, 8, s));
      DG_CUDA(dg::launch_lca(p, mode, c, s));
      return DG_OK;
    };
    if (mode == DG_MODE_PLAIN) return go(dg::LaunchCfg{});
    auto cands = lca_candidates(m->N, d->n_trials, lpt);
    if (cands.empty()) return fail(DG_E_UNSUPPORTED, "dg_run: no LCA layout for N=%d", m->N);
    return run_tuned(m->ctx,
                     "lca" + std::to_string(m->N) + "/" + bucket + "/t" +
                         std::to_string(forced_tpt()) + "/o" + std::to_string(forced_order()),
                     cands, s, go);
  }
  if (m->kind == K_NET) {
    dg::NetParams p{};
    p.layout = m->d_layout;
    p.w_in = m->d_w_in;
    p.cond = d->cond_inputs;
    p.n_cond = d->n_cond;
    p.cond_block = d->cond_block;
    p.n = d->n_trials;
    p.trial0 = (uint32_t)d->trial_offset;
    p.k0 = k0;
    p.k1 = k1;
    p.rk = dg::philox_keys(k0, k1);
    p.U = m->layout.U;
    p.n_in = m->layout.n_in;
    p.stop_size = m->layout.stop_size;
    p.n_ddm = m->layout.n_ddm;
    p.state_size = m->state_size;
    p.choice = choice;
    p.step = step;
    p.yout = fs;
    p.cursor = mode == DG_MODE_BATCHED ? sc->cursor() : nullptr;
    if (mode == DG_MODE_BATCHED) DG_CUDA(cudaMemsetAsync(sc->cursor(), 0, 8, s));
    if (mode == DG_MODE_BATCHED && m->layout.U <= dg::kLaneMaxU && net_lane_enabled()) {
      DG_CUDA(dg::launch_net_lane(p, net_dense(m->layout), s));
      return DG_OK;
    }
    DG_CUDA(dg::launch_net(p, mode, dg::LaunchCfg{}, s));
    return DG_OK;
  }
  if (m->kind == K_WIDE) {
    dg::WideParams p{};
    p.w_in = m->d_w_hid;
    p.w_resp_bf16 = m->d_w_resp_bf16;
    p.w_resp_f32 = m->d_w_resp_f32;
    p.cond = d->cond_inputs;
    p.n_cond = d->n_cond;
    p.cond_block = d->cond_block;
    p.S = m->S;
    p.T = m->T;
    p.H = m->H;
    p.R = m->R;
    p.bias_h = m->bias_h;
    p.bias_r = m->bias_r;
    p.gain_h = m->gain_h;
    p.gain_r = m->gain_r;
    p.rate = m->rate;
    p.noise = m->noise;
    p.stop_threshold = m->stop_thr;
    p.max_steps = m->max_steps;
    p.n = d->n_trials;
    p.trial0 = (uint32_t)d->trial_offset;
    p.k0 = k0;
    p.k1 = k1;
    p.rk = dg::philox_keys(k0, k1);
    p.choice = choice;
    p.step = step;
    p.yout = fs;
    p.cursor = sc->cursor();
    p.status = sc->status();
    if (mode == DG_MODE_BATCHED) {
      // hidden net input of each condition (H floats per condition)
      if ((st = scratch_net(m->ctx, sc, (size_t)d->n_cond * m->H, s)) != DG_OK) return st;
      p.net_table = sc->net;
    }
    DG_CUDA(cudaMemsetAsync(sc->cursor(), 0, 8, s));
    cudaError_t e = dg::launch_wide(p, mode, dg::LaunchCfg{}, s);
    if (e == cudaErrorNotSupported)
      return fail(DG_E_UNSUPPORTED, "wide network kernel not available in this build");
    DG_CUDA(e);
    return DG_OK;
  }
  return fail(DG_E_UNSUPPORTED, "dg_run: predator-prey models run through dg_grid_search");
}

dg_status check_run_args(dg_model* m, const dg_run_desc* d, int8_t* choice, int32_t* step) {
  if (!m || !d) return fail(DG_E_ARG, "dg_run: null model or desc");
  if (d->n_trials < 0 || d->n_trials > INT32_MAX)
    return fail(DG_E_ARG, "dg_run: n_trials %lld out of range [0, 2^31-1]", (long long)d->n_trials);
  if (d->mode != DG_MODE_BATCHED && d->mode != DG_MODE_PLAIN)
    return fail(DG_E_ARG, "dg_run: unknown mode %d", d->mode);
  if (d->trial_offset < 0 || d->trial_offset + d->n_trials > (1ll << 32))
    return fail(DG_E_ARG, "dg_run: trial_offset + n_trials must lie in [0, 2^32]");
  if (m->kind == K_PP)
    return fail(DG_E_UNSUPPORTED, "dg_run: predator-prey models run through dg_grid_search");
  if (d->n_trials == 0) return DG_OK;
  if (!choice || !step) return fail(DG_E_ARG, "dg_run: null choice or step output");
  if ((m->kind == K_DDM || m->kind == K_LCA) && !d->trial_params)
    return fail(DG_E_ARG, "dg_run: trial_params required for DDM and LCA models");
  if (m->kind == K_NET || m->kind == K_WIDE) {
    if (!d->cond_inputs) return fail(DG_E_ARG, "dg_run: cond_inputs required");
    if (d->n_cond < 1 || d->cond_block < 1)
      return fail(DG_E_ARG, "dg_run: n_cond and cond_block must be >= 1");
  }
  return DG_OK;
}

size_t run_param_floats(const dg_model* m, const dg_run_desc* d) {
  if (m->kind == K_DDM) return 2 * (size_t)d->n_trials;
  if (m->kind == K_LCA) return (size_t)d->n_trials * m->N;
  return 0;
}

size_t run_cond_floats(const dg_model* m, const dg_run_desc* d) {
  if (m->kind == K_NET || m->kind == K_WIDE) return (size_t)d->n_cond * m->n_inputs;
  return 0;
}

// Several jobs of one DDM or LCA model in one persistent launch: the jobs'
// trials form one list (job i's trials after those of jobs 0 .. i-1, empty
// jobs left out) that the kernel hands out from one cursor; each trial runs
// with its job's inputs, outputs, seed and trial offset, exactly as in a
// batched dg_run of that job alone. Arguments are checked by the caller.
dg_status run_jobs_device(dg_model* m, int n_jobs, const dg_run_desc* d, int8_t* const* choice,
                          int32_t* const* step, float* const* fs, cudaStream_t s) {
  dg::MultiJobTable tab{};
  long long total = 0;
  for (int i = 0; i < n_jobs; ++i) {
    if (d[i].n_trials == 0) continue;
    dg::MultiJob& J = tab.jobs[tab.n_jobs++];
    J.start = total;
    J.n = d[i].n_trials;
    J.in = m->kind == K_NET ? d[i].cond_inputs : d[i].trial_params;
    J.n_cond = d[i].n_cond;
    J.cond_block = d[i].cond_block;
    J.choice = choice[i];
    J.step = step[i];
    J.xout = fs ? fs[i] : nullptr;
    J.trial0 = (uint32_t)d[i].trial_offset;
    J.k0 = (uint32_t)d[i].seed;
    J.k1 = (uint32_t)(d[i].seed >> 32);
    total += d[i].n_trials;
  }
  if (total == 0) return DG_OK;
  Scratch* sc = nullptr;
  dg_status st = get_scratch(m->ctx, s, &sc);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemsetAsync(sc->cursor(), 0, 8, s));
  if (m->kind == K_DDM) {
    dg::DdmParams p = ddm_model_params(m);
    p.n = total;
    p.cursor = sc->cursor();
    DG_CUDA(dg::launch_ddm_multi(p, tab, s));
    return DG_OK;
  }
  if (m->kind == K_NET) {
    dg::NetParams p{};
    p.layout = m->d_layout;
    p.w_in = m->d_w_in;
    p.n = total;
    p.U = m->layout.U;
    p.n_in = m->layout.n_in;
    p.stop_size = m->layout.stop_size;
    p.n_ddm = 0;
    p.state_size = m->state_size;
    p.cursor = sc->cursor();
    DG_CUDA(dg::launch_net_lane_multi(p, net_dense(m->layout), tab, s));
    return DG_OK;
  }
  dg::LcaParams p = lca_model_params(m);
  p.n = total;
  p.cursor = sc->cursor();
  DG_CUDA(dg::launch_lca_multi(p, tab, s));
  return DG_OK;
}

dg_status check_jobs_args(dg_model* m, int n_jobs, const dg_run_desc* d, int8_t* const* choice,
                          int32_t* const* step) {
  if (!m || !d || !choice || !step || n_jobs < 1 || n_jobs > dg::kMaxMultiJobs)
    return fail(DG_E_ARG, "dg_run_jobs: null model, descs or outputs, or n_jobs outside [1, %d]",
                dg::kMaxMultiJobs);
  if (m->kind != K_DDM && m->kind != K_LCA && !net_lane_model(m))
    return fail(DG_E_UNSUPPORTED, "dg_run_jobs: DDM, LCA and small network models only "
                                  "(at most %d logistic units, no DDM nodes)", dg::kLaneMaxU);
  long long total = 0;
  for (int i = 0; i < n_jobs; ++i) {
    dg_status st = check_run_args(m, d + i, choice[i], step[i]);
    if (st != DG_OK) return st;
    if (d[i].mode != DG_MODE_BATCHED)
      return fail(DG_E_ARG, "dg_run_jobs: job %d: the batched mode only", i);
    total += d[i].n_trials;
  }
  if (total > INT32_MAX)
    return fail(DG_E_ARG, "dg_run_jobs: %lld trials in all, at most 2^31-1", total);
  return DG_OK;
}

// ------------------------------------------------------------- grid ---

dg_status check_grid_args(dg_model* m, const dg_grid_desc* d, dg_grid_result* result) {
  if (!m || !d || !result) return fail(DG_E_ARG, "dg_grid_search: null model, desc or result");
  if (m->kind != K_PP)
    return fail(DG_E_UNSUPPORTED, "dg_grid_search: model is not a predator-prey model");
  for (int i = 0; i < 3; ++i)
    if (d->n_levels[i] < 1 || d->n_levels[i] > 4096)
      return fail(DG_E_ARG, "dg_grid_search: n_levels[%d] = %d out of [1, 4096]", i,
                  d->n_levels[i]);
  if (d->n_trials < 1 || d->n_trials > 1024)
    return fail(DG_E_ARG, "dg_grid_search: n_trials %d out of [1, 1024]", d->n_trials);
  if (!d->positions || !d->levels[0] || !d->levels[1] || !d->levels[2])
    return fail(DG_E_ARG, "dg_grid_search: null positions or levels");
  if (d->mode != DG_MODE_BATCHED && d->mode != DG_MODE_PLAIN)
    return fail(DG_E_ARG, "dg_grid_search: unknown mode %d", d->mode);
  if (d->tie_break != DG_TIE_LOWEST && d->tie_break != DG_TIE_RESERVOIR)
    return fail(DG_E_ARG, "dg_grid_search: unknown tie_break %d", d->tie_break);
  const long long n = (long long)d->n_levels[0] * d->n_levels[1] * d->n_levels[2];
  if (n > 0xFFFFFFFFll) return fail(DG_E_ARG, "dg_grid_search: more than 2^32 candidates");
  if (d->cand_begin < 0 || d->cand_count < 0 || d->cand_begin + d->cand_count > n ||
      (d->cand_count == 0 && d->cand_begin != 0))
    return fail(DG_E_ARG, "dg_grid_search: candidate range [%lld, +%lld) outside [0, %lld)",
                (long long)d->cand_begin, (long long)d->cand_count, n);
  return DG_OK;
}

dg_status grid_device(dg_model* m, const dg_grid_desc* d, dg_grid_result* result, double* means,
                      cudaStream_t s) {
  Scratch* sc = nullptr;
  dg_status st = get_scratch(m->ctx, s, &sc);
  if (st != DG_OK) return st;
  dg::GridParams p{};
  for (int i = 0; i < 3; ++i) {
    p.lv[i] = d->levels[i];
    p.L[i] = d->n_levels[i];
  }
  p.pos = d->positions;
  p.n_trials = d->n_trials;
  p.k0 = (uint32_t)d->seed;
  p.k1 = (uint32_t)(d->seed >> 32);
  p.rk = dg::philox_keys(p.k0, p.k1);
  p.offset = m->offset;
  p.weight = m->weight;
  const long long total = (long long)d->n_levels[0] * d->n_levels[1] * d->n_levels[2];
  p.cand0 = d->cand_begin;
  p.n_cand = d->cand_count ? d->cand_count : total;
  p.means = means;
  p.partials = sc->partials();
  p.ticket = sc->ticket();
  p.result = result;
  const bool reservoir = d->tie_break == DG_TIE_RESERVOIR;
  if ((d->mode == DG_MODE_PLAIN || reservoir) && !means) {
    st = scratch_means(m->ctx, sc, (size_t)p.n_cand, s);
    if (st != DG_OK) return st;
    p.means = sc->means;
  }
  auto go = [&](const dg::LaunchCfg& c) -> dg_status {
    DG_CUDA(cudaMemsetAsync(sc->ticket(), 0, 4, s));
    DG_CUDA(dg::launch_grid(p, d->mode, c, s));
    if (reservoir)
      DG_CUDA(dg::launch_tie_reservoir(p.means, p.n_cand, p.cand0, d->seed, result, s));
    return DG_OK;
  };
  if (d->mode == DG_MODE_PLAIN) return go(dg::LaunchCfg{});
  const std::string key = "grid/" + std::to_string(log2_bucket(p.n_cand)) + "/" +
                          std::to_string(log2_bucket(p.n_trials));
  return run_tuned(m->ctx, key, grid_candidates(p.n_cand, dg::grid_lanes(p.L)), s, go);
}

dg_status check_grid_batch(dg_model* m, int32_t n_searches, const dg_grid_desc* descs,
                           const dg_grid_result* results) {
  if (!m || !descs || !results || n_searches < 1 || n_searches > dg::kMaxGridBatch)
    return fail(DG_E_ARG, "dg_grid_search_batch: null model, descs or results, or n_searches "
                          "outside [1, %d]", dg::kMaxGridBatch);
  for (int i = 0; i < n_searches; ++i) {
    const dg_grid_desc& d = descs[i];
    dg_status st = check_grid_args(m, &d, const_cast<dg_grid_result*>(results));
    if (st != DG_OK) return st;
    for (int e = 0; e < 3; ++e)
      if (d.n_levels[e] != descs[0].n_levels[e])
        return fail(DG_E_ARG, "dg_grid_search_batch: search %d has another grid shape", i);
    if (d.n_trials != descs[0].n_trials)
      return fail(DG_E_ARG, "dg_grid_search_batch: search %d has another trial count", i);
    if (d.cand_begin != 0 || d.cand_count != 0 || d.tie_break != DG_TIE_LOWEST ||
        d.mode != DG_MODE_BATCHED)
      return fail(DG_E_ARG, "dg_grid_search_batch: search %d: whole grids, lowest-index ties "
                            "and the batched mode only", i);
  }
  return DG_OK;
}

// A checked batch of whole-grid searches of one shape in one launch; search i
// writes results[i] and, when not null, cand_means[i].
dg_status grid_batch_device(dg_model* m, int32_t n_searches, const dg_grid_desc* descs,
                            dg_grid_result* const* results, double* const* cand_means,
                            cudaStream_t s) {
  Scratch* sc = nullptr;
  dg_status st = get_scratch(m->ctx, s, &sc);
  if (st != DG_OK) return st;
  dg::GridBatchParams p{};
  for (int e = 0; e < 3; ++e) p.L[e] = descs[0].n_levels[e];
  p.n_trials = descs[0].n_trials;
  p.offset = m->offset;
  p.weight = m->weight;
  p.n_cand = (long long)p.L[0] * p.L[1] * p.L[2];
  p.cpc = (int)((p.n_cand + dg::kGridChunk - 1) / dg::kGridChunk);
  p.n_search = n_searches;
  const size_t head = 256 + ((size_t)n_searches * sizeof(unsigned int) + 255) / 256 * 256;
  const size_t bytes = head + (size_t)n_searches * p.cpc * sizeof(dg::TopTwo);
  if ((st = scratch_gb(m->ctx, sc, bytes, s)) != DG_OK) return st;
  p.cursor = reinterpret_cast<unsigned long long*>(sc->gb);
  p.ticket = reinterpret_cast<unsigned int*>(sc->gb + 256);
  p.partials = reinterpret_cast<dg::TopTwo*>(sc->gb + head);
  for (int i = 0; i < n_searches; ++i) {
    dg::GridBatchItem& it = p.items[i];
    for (int e = 0; e < 3; ++e) it.lv[e] = descs[i].levels[e];
    it.pos = descs[i].positions;
    it.result = results[i];
    it.means = cand_means ? cand_means[i] : nullptr;
    it.k0 = (uint32_t)descs[i].seed;
    it.k1 = (uint32_t)(descs[i].seed >> 32);
  }
  DG_CUDA(cudaMemsetAsync(sc->gb, 0, head, s));
  DG_CUDA(dg::launch_grid_batch(p, s));
  return DG_OK;
}

// ------------------------------------------------------------ serving ---

struct JobRec {
  uint64_t id = 0;
  dg_job job{};
  dg_status status = DG_OK;
  int state = 0;  // 0 queued, 1 running, 2 done
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int slot = -1;
  void* dmem = nullptr;
};

struct Server {
  dg_ctx* ctx;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::shared_ptr<JobRec>> jobs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<std::vector<uint64_t>> slot_jobs;  // the jobs of the slot's launch; empty = free
  size_t in_use = 0;
  // Small DDM and LCA jobs of one model share one launch (dg_run_jobs): a
  // job of at most group_job_trials trials gathers later queued jobs of the
  // same model, up to kMaxMultiJobs jobs and kGroupTrials trials in all.
  long long group_job_trials = 1 << 16;
  static constexpr long long kGroupTrials = 1 << 23;
  // Grouped jobs whose host buffers are pinned (mapped into the device's
  // address space) are read and written by the kernel in place, over the
  // host link, with no staging copies.
  bool zero_copy = true;
  static constexpr size_t kGroupScan = 4096;   // queued jobs looked at per group
  uint64_t next_id = 1;
  int64_t n_running = 0, n_done = 0;
  bool stop = false;
  std::thread th;

  explicit Server(dg_ctx* c, int slots) : ctx(c) {
    cudaSetDevice(ctx->device);
    // Job memory comes from the stream-ordered allocator: allocation and
    // release are ordered on the job's stream and never synchronize the
    // device, so admitted jobs keep overlapping. The pool keeps freed memory
    // for reuse instead of returning it to the CUDA driver.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int i = 0; i < slots; ++i) {
      cudaStream_t s;
      cudaEvent_t e;
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      streams.push_back(s);
      events.push_back(e);
      slot_jobs.emplace_back();
    }
    if (const char* e = getenv("DG_SERVE_GROUP_TRIALS")) group_job_trials = atoll(e);
    if (const char* e = getenv("DG_SERVE_ZERO_COPY")) zero_copy = atoi(e) != 0;
    th = std::thread([this] { loop(); });
  }

  ~Server() {
    {
      std::lock_guard<std::mutex> g(mu);
      stop = true;
    }
    cv_work.notify_all();
    if (th.joinable()) th.join();
    for (auto s : streams) cudaStreamSynchronize(s);
    for (auto& kv : jobs)
      if (kv.second->dmem) cudaFree(kv.second->dmem);
    cudaDeviceSynchronize();
    for (auto s : streams) cudaStreamDestroy(s);
    for (auto e : events) cudaEventDestroy(e);
  }

  static size_t job_bytes(const dg_job& j) {
    size_t b = 1024;  // alignment slack
    if (j.is_grid) {
      const size_t nc = j.grid.cand_count ? (size_t)j.grid.cand_count
                                          : (size_t)j.grid.n_levels[0] * j.grid.n_levels[1] *
                                                j.grid.n_levels[2];
      b += 6 * sizeof(float) * (size_t)j.grid.n_trials;
      b += sizeof(float) * ((size_t)j.grid.n_levels[0] + j.grid.n_levels[1] + j.grid.n_levels[2]);
      b += sizeof(dg_grid_result) + sizeof(double) * nc;
    } else {
      const size_t n = (size_t)j.run.n_trials;
      b += sizeof(float) * (run_param_floats(j.model, &j.run) + run_cond_floats(j.model, &j.run));
      b += n * (sizeof(int8_t) + sizeof(int32_t));
      if (j.final_state) b += n * sizeof(float) * (size_t)j.model->state_size;
    }
    return b + 16 * 256;
  }

  static long long grid_cands(const dg_grid_desc& g) {
    return (long long)g.n_levels[0] * g.n_levels[1] * g.n_levels[2];
  }

  // Jobs that can share a launch with others: runs of a job-table model up to
  // group_job_trials trials; whole-grid searches (lowest-index ties) up to as
  // many candidates.
  bool groupable(const JobRec& r) const {
    const dg_job& j = r.job;
    if (j.is_grid)
      return j.model->kind == K_PP && j.grid.mode == DG_MODE_BATCHED &&
             j.grid.tie_break == DG_TIE_LOWEST && j.grid.cand_begin == 0 &&
             j.grid.cand_count == 0 && grid_cands(j.grid) <= group_job_trials;
    return (j.model->kind == K_DDM || j.model->kind == K_LCA || net_lane_model(j.model)) &&
           j.run.mode == DG_MODE_BATCHED && j.run.n_trials > 0 &&
           j.run.n_trials <= group_job_trials;
  }

  // b may join a's launch: the same model, and for searches the same grid
  // shape and trial count.
  static bool same_group(const dg_job& a, const dg_job& b) {
    if (a.model != b.model || a.is_grid != b.is_grid) return false;
    if (!a.is_grid) return true;
    for (int e = 0; e < 3; ++e)
      if (a.grid.n_levels[e] != b.grid.n_levels[e]) return false;
    return a.grid.n_trials == b.grid.n_trials;
  }

  // Device copies of a run job: inputs copied in, outputs allocated.
  struct Staged {
    dg_run_desc d;
    int8_t* choice;
    int32_t* step;
    float* fs;
  };

  dg_status stage_run(JobRec& r, cudaStream_t s, Staged* out) {
    DG_CUDA(cudaMallocAsync(&r.dmem, r.bytes, s));
    unsigned char* p = reinterpret_cast<unsigned char*>(r.dmem);
    auto take = [&](size_t bytes) {
      unsigned char* q = p;
      p += (bytes + 255) / 256 * 256;
      return q;
    };
    const dg_job& j = r.job;
    dg_run_desc d = j.run;
    const size_t n = (size_t)d.n_trials;
    const size_t pf = run_param_floats(j.model, &d), cf = run_cond_floats(j.model, &d);
    if (pf) {
      float* tp = (float*)take(pf * sizeof(float));
      DG_CUDA(cudaMemcpyAsync(tp, j.run.trial_params, pf * sizeof(float), cudaMemcpyHostToDevice, s));
      d.trial_params = tp;
    }
    if (cf) {
      float* ci = (float*)take(cf * sizeof(float));
      DG_CUDA(cudaMemcpyAsync(ci, j.run.cond_inputs, cf * sizeof(float), cudaMemcpyHostToDevice, s));
      d.cond_inputs = ci;
    }
    out->d = d;
    out->choice = (int8_t*)take(n);
    out->step = (int32_t*)take(n * sizeof(int32_t));
    out->fs = j.final_state ? (float*)take(n * sizeof(float) * j.model->state_size) : nullptr;
    return DG_OK;
  }

  dg_status unstage_run(JobRec& r, cudaStream_t s, const Staged& g) {
    const dg_job& j = r.job;
    const size_t n = (size_t)j.run.n_trials;
    DG_CUDA(cudaMemcpyAsync(j.choice, g.choice, n, cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaMemcpyAsync(j.step, g.step, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (g.fs)
      DG_CUDA(cudaMemcpyAsync(j.final_state, g.fs, n * sizeof(float) * j.model->state_size,
                              cudaMemcpyDeviceToHost, s));
    return DG_OK;
  }

  // The device address of pinned, mapped host memory; null for anything else
  // (pageable memory, device memory, an unknown pointer).
  static void* mapped_alias(const void* h) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
      cudaGetLastError();   // not a pointer the runtime knows: clear the error it left
      return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
  }

  // A run job's buffers as the kernel can use them in place, if all are
  // pinned and mapped.
  static bool in_place(const dg_job& j, Staged* out) {
    const bool net = j.model->kind == K_NET;
    const float* in = (const float*)mapped_alias(net ? j.run.cond_inputs : j.run.trial_params);
    int8_t* ch = (int8_t*)mapped_alias(j.choice);
    int32_t* st = (int32_t*)mapped_alias(j.step);
    float* fs = j.final_state ? (float*)mapped_alias(j.final_state) : nullptr;
    if (!in || !ch || !st || (j.final_state && !fs)) return false;
    out->d = j.run;
    if (net)
      out->d.cond_inputs = in;
    else
      out->d.trial_params = in;
    out->choice = ch;
    out->step = st;
    out->fs = fs;
    return true;
  }

  // Enqueue a group's copies (for jobs not used in place) and one multi-job
  // launch on its slot's stream.
  dg_status launch_group(const std::vector<std::shared_ptr<JobRec>>& grp, cudaStream_t s) {
    const int n = (int)grp.size();
    std::vector<Staged> g(n);
    std::vector<char> direct(n, 0);
    std::vector<dg_run_desc> d(n);
    std::vector<int8_t*> ch(n);
    std::vector<int32_t*> stp(n);
    std::vector<float*> fs(n);
    for (int i = 0; i < n; ++i) {
      direct[i] = zero_copy && in_place(grp[i]->job, &g[i]);
      if (!direct[i]) {
        dg_status st = stage_run(*grp[i], s, &g[i]);
        if (st != DG_OK) return st;
      }
      d[i] = g[i].d;
      ch[i] = g[i].choice;
      stp[i] = g[i].step;
      fs[i] = g[i].fs;
    }
    dg_status st = run_jobs_device(grp[0]->job.model, n, d.data(), ch.data(), stp.data(),
                                   fs.data(), s);
    if (st != DG_OK) return st;
    for (int i = 0; i < n; ++i)
      if (!direct[i] && (st = unstage_run(*grp[i], s, g[i])) != DG_OK) return st;
    return DG_OK;
  }

  // Enqueue a group of searches of one grid shape: each job's positions and
  // levels copied in, one batched launch, each job's result (and means) out.
  dg_status launch_grid_group(const std::vector<std::shared_ptr<JobRec>>& grp, cudaStream_t s) {
    const int n = (int)grp.size();
    std::vector<dg_grid_desc> d(n);
    std::vector<dg_grid_result*> res(n);
    std::vector<double*> means(n);
    for (int i = 0; i < n; ++i) {
      JobRec& r = *grp[i];
      const dg_job& j = r.job;
      DG_CUDA(cudaMallocAsync(&r.dmem, r.bytes, s));
      unsigned char* p = reinterpret_cast<unsigned char*>(r.dmem);
      auto take = [&](size_t bytes) {
        unsigned char* q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
      };
      d[i] = j.grid;
      float* pos = (float*)take(6 * sizeof(float) * d[i].n_trials);
      DG_CUDA(cudaMemcpyAsync(pos, j.grid.positions, 6 * sizeof(float) * d[i].n_trials,
                              cudaMemcpyHostToDevice, s));
      d[i].positions = pos;
      for (int e = 0; e < 3; ++e) {
        float* lv = (float*)take(sizeof(float) * d[i].n_levels[e]);
        DG_CUDA(cudaMemcpyAsync(lv, j.grid.levels[e], sizeof(float) * d[i].n_levels[e],
                                cudaMemcpyHostToDevice, s));
        d[i].levels[e] = lv;
      }
      res[i] = (dg_grid_result*)take(sizeof(dg_grid_result));
      means[i] = (double*)take(sizeof(double) * (size_t)grid_cands(d[i]));
    }
    dg_status st = grid_batch_device(grp[0]->job.model, n, d.data(), res.data(), means.data(), s);
    if (st != DG_OK) return st;
    for (int i = 0; i < n; ++i) {
      const dg_job& j = grp[i]->job;
      DG_CUDA(cudaMemcpyAsync(j.grid_result, res[i], sizeof(dg_grid_result),
                              cudaMemcpyDeviceToHost, s));
      if (j.cand_means)
        DG_CUDA(cudaMemcpyAsync(j.cand_means, means[i], sizeof(double) * (size_t)grid_cands(d[i]),
                                cudaMemcpyDeviceToHost, s));
    }
    return DG_OK;
  }

  // Enqueue a job's copies and kernels on its slot's stream.
  dg_status launch(JobRec& r, cudaStream_t s) {
    const dg_job& j = r.job;
    if (!j.is_grid) {
      Staged g;
      dg_status st = stage_run(r, s, &g);
      if (st != DG_OK) return st;
      if ((st = run_device(j.model, &g.d, g.choice, g.step, g.fs, s)) != DG_OK) return st;
      return unstage_run(r, s, g);
    }
    DG_CUDA(cudaMallocAsync(&r.dmem, r.bytes, s));
    unsigned char* p = reinterpret_cast<unsigned char*>(r.dmem);
    auto take = [&](size_t bytes) {
      unsigned char* q = p;
      p += (bytes + 255) / 256 * 256;
      return q;
    };
    dg_grid_desc d = j.grid;
    const size_t nc = d.cand_count ? (size_t)d.cand_count
                                   : (size_t)d.n_levels[0] * d.n_levels[1] * d.n_levels[2];
    float* pos = (float*)take(6 * sizeof(float) * d.n_trials);
    DG_CUDA(cudaMemcpyAsync(pos, j.grid.positions, 6 * sizeof(float) * d.n_trials,
                            cudaMemcpyHostToDevice, s));
    d.positions = pos;
    for (int i = 0; i < 3; ++i) {
      float* lv = (float*)take(sizeof(float) * d.n_levels[i]);
      DG_CUDA(cudaMemcpyAsync(lv, j.grid.levels[i], sizeof(float) * d.n_levels[i],
                              cudaMemcpyHostToDevice, s));
      d.levels[i] = lv;
    }
    dg_grid_result* res = (dg_grid_result*)take(sizeof(dg_grid_result));
    double* means = (double*)take(sizeof(double) * nc);
    dg_status st = grid_device(j.model, &d, res, means, s);
    if (st != DG_OK) return st;
    DG_CUDA(cudaMemcpyAsync(j.grid_result, res, sizeof(dg_grid_result),
                            cudaMemcpyDeviceToHost, s));
    if (j.cand_means)
      DG_CUDA(cudaMemcpyAsync(j.cand_means, means, sizeof(double) * nc,
                              cudaMemcpyDeviceToHost, s));
    return DG_OK;
  }

  void finish(JobRec& r, dg_status st) {
    if (r.dmem) {
      // the job's stream has passed its completion event, so this is ordered
      // after every use of the memory
      cudaFreeAsync(r.dmem, r.slot >= 0 ? streams[r.slot] : nullptr);
      r.dmem = nullptr;
    }
    in_use -= r.bytes;
    r.status = st;
    r.state = 2;
    r.t_done = now_s();
    r.slot = -1;
    --n_running;
    ++n_done;
  }

  void loop() {
    cudaSetDevice(ctx->device);
    t_no_tune = true;
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progress = false;
      // retire finished jobs
      for (size_t i = 0; i < streams.size(); ++i) {
        if (slot_jobs[i].empty()) continue;
        cudaError_t q = cudaEventQuery(events[i]);
        if (q == cudaErrorNotReady) continue;
        for (uint64_t id : slot_jobs[i]) finish(*jobs[id], q == cudaSuccess ? DG_OK : DG_E_CUDA);
        slot_jobs[i].clear();
        progress = true;
      }
      if (progress) cv_done.notify_all();
      // admit queued jobs in arrival order while memory and slots allow;
      // the launches themselves happen without the lock
      std::vector<std::vector<std::shared_ptr<JobRec>>> admitted;
      while (!queue.empty()) {
        auto rp = jobs[queue.front()];
        if (in_use + rp->bytes > ctx->budget) break;
        int slot = -1;
        for (size_t i = 0; i < streams.size(); ++i)
          if (slot_jobs[i].empty()) {
            slot = (int)i;
            break;
          }
        if (slot < 0) break;
        queue.pop_front();
        std::vector<std::shared_ptr<JobRec>> grp{rp};
        size_t bytes = rp->bytes;
        if (groupable(*rp)) {
          const bool grid = rp->job.is_grid;
          const int max_jobs = grid ? dg::kMaxGridBatch : dg::kMaxMultiJobs;
          auto units = [&](const JobRec& r) {   // trials, or candidate evaluations
            return grid ? grid_cands(r.job.grid) * r.job.grid.n_trials : r.job.run.n_trials;
          };
          long long total = units(*rp);
          size_t scanned = 0;
          for (auto it = queue.begin();
               it != queue.end() && scanned < kGroupScan && (int)grp.size() < max_jobs;
               ++scanned) {
            auto& q = jobs[*it];
            if (groupable(*q) && same_group(rp->job, q->job) &&
                total + units(*q) <= (grid ? 64 * kGroupTrials : kGroupTrials) &&
                in_use + bytes + q->bytes <= ctx->budget) {
              grp.push_back(q);
              total += units(*q);
              bytes += q->bytes;
              it = queue.erase(it);
            } else {
              ++it;
            }
          }
        }
        const double t = now_s();
        for (auto& g : grp) {
          g->slot = slot;
          g->state = 1;
          g->t_admit = t;
          in_use += g->bytes;
          ++n_running;
          slot_jobs[slot].push_back(g->id);
        }
        admitted.push_back(std::move(grp));
      }
      if (!admitted.empty()) {
        progress = true;
        lk.unlock();
        std::vector<std::pair<std::shared_ptr<JobRec>, dg_status>> failed;
        for (auto& grp : admitted) {
          const int slot = grp[0]->slot;
          cudaStream_t s = streams[slot];
          dg_status st = grp.size() == 1      ? launch(*grp[0], s)
                         : grp[0]->job.is_grid ? launch_grid_group(grp, s)
                                               : launch_group(grp, s);
          if (st == DG_OK && cudaEventRecord(events[slot], s) != cudaSuccess) st = DG_E_CUDA;
          if (st != DG_OK) {
            cudaStreamSynchronize(s);
            for (auto& g : grp) failed.emplace_back(g, st);
          }
        }
        lk.lock();
        for (auto& f : failed) {
          const int slot = f.first->slot;
          finish(*f.first, f.second);
          if (slot >= 0) slot_jobs[slot].clear();
        }
        if (!failed.empty()) cv_done.notify_all();
      }
      if (stop) break;
      if (!progress) {
        if (n_running > 0)
          cv_work.wait_for(lk, std::chrono::microseconds(50));
        else
          cv_work.wait_for(lk, std::chrono::milliseconds(5));
      }
    }
  }
};

Server* server_of(dg_ctx* ctx) {
  std::lock_guard<std::mutex> g(ctx->server_mu);
  if (!ctx->server) {
    int slots = 16;
    if (const char* e = getenv("DG_SERVE_SLOTS")) slots = std::max(1, atoi(e));
    ctx->server.reset(new Server(ctx, slots));
  }
  return ctx->server.get();
}

// ------------------------------------------------------------ compose ---

uint16_t to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;  // round to nearest even
  return (uint16_t)(u >> 16);
}

float from_bf16(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

template <class T>
dg_status upload(T** dst, const std::vector<T>& v) {
  DG_CUDA(cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!v.empty()) DG_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DG_OK;
}

dg_status compose_transfer(dg_model* m, const dg_mechanism* mechs, int n_mech,
                           const dg_projection* projs, int n_proj, const dg_stop* stop) {
  std::vector<int> noff(n_mech, -1), ioff(n_mech, -1), doff(n_mech, -1);
  int U = 0, n_in = 0, n_logistic = 0, n_ddm = 0;
  for (int i = 0; i < n_mech; ++i) {
    if (mechs[i].kind == DG_INPUT) {
      ioff[i] = n_in;
      n_in += mechs[i].size;
    } else if (mechs[i].kind == DG_DDM) {
      doff[i] = n_ddm;
      n_ddm += mechs[i].size;
    } else if (mechs[i].kind == DG_TRANSFER_LOGISTIC) {
      noff[i] = U;
      U += mechs[i].size;
      ++n_logistic;
    } else {
      return fail(DG_E_SHAPE, "compose: mechanism %d cannot be part of a transfer network", i);
    }
  }
  if (n_ddm > dg::kNetMaxDdm)
    return fail(DG_E_UNSUPPORTED, "compose: at most %d DDM units on the stop layer", dg::kNetMaxDdm);
  if (n_logistic == 0) return fail(DG_E_SHAPE, "compose: no logistic layer");
  if (stop->mech < 0 || stop->mech >= n_mech || mechs[stop->mech].kind != DG_TRANSFER_LOGISTIC)
    return fail(DG_E_SHAPE, "compose: stop mechanism must be a logistic layer");
  if (mechs[stop->mech].size < 2 || mechs[stop->mech].size > 16)
    return fail(DG_E_SHAPE, "compose: stop layer needs 2..16 units");
  double rate = -1, noise = -1;
  for (int i = 0; i < n_mech; ++i) {
    if (mechs[i].kind != DG_TRANSFER_LOGISTIC) continue;
    if (!(mechs[i].rate > 0.0 && mechs[i].rate <= 1.0))
      return fail(DG_E_ARG, "compose: mechanism %d rate must be in (0, 1]", i);
    if (!(mechs[i].noise >= 0.0)) return fail(DG_E_ARG, "compose: mechanism %d noise < 0", i);
    if (rate < 0) {
      rate = mechs[i].rate;
      noise = mechs[i].noise;
    } else if (rate != mechs[i].rate || noise != mechs[i].noise) {
      return fail(DG_E_UNSUPPORTED, "compose: all logistic layers must share rate and noise");
    }
  }
  for (int p = 0; p < n_proj; ++p) {
    const auto& e = projs[p];
    if (e.sender < 0 || e.sender >= n_mech || e.receiver < 0 || e.receiver >= n_mech)
      return fail(DG_E_SHAPE, "compose: projection %d has an invalid endpoint", p);
    if (mechs[e.sender].kind == DG_DDM)
      return fail(DG_E_SHAPE, "compose: projection %d leaves a DDM node (DDM nodes send nothing)", p);
    if (mechs[e.receiver].kind == DG_DDM) {
      if (e.sender != stop->mech || e.dtype != DG_F32)
        return fail(DG_E_SHAPE, "compose: DDM node inputs are F32 projections from the stop layer (projection %d)", p);
    } else if (mechs[e.receiver].kind != DG_TRANSFER_LOGISTIC) {
      return fail(DG_E_SHAPE, "compose: projection %d must end at a logistic layer", p);
    }
    if (!e.weights) return fail(DG_E_ARG, "compose: projection %d has no weights", p);
    if (e.dtype != DG_F32 && e.dtype != DG_BF16)
      return fail(DG_E_ARG, "compose: projection %d has unknown dtype", p);
  }
  for (int i = 0; i < n_mech; ++i) {
    if (mechs[i].kind != DG_DDM) continue;
    const auto& g = mechs[i];
    if (!(g.dt > 0.0) || !(g.noise >= 0.0) || !(g.threshold > 0.0) || g.max_steps < 1 ||
        g.start != 0.0)
      return fail(DG_E_ARG, "compose: DDM node %d needs dt > 0, noise >= 0, threshold > 0, "
                  "max_steps >= 1 and start 0", i);
  }
  m->max_steps = stop->max_steps;
  m->state_size = mechs[stop->mech].size + 3 * n_ddm;
  m->n_inputs = n_in;
  m->rate = (float)rate;
  m->noise = (float)noise;
  m->stop_thr = (float)stop->threshold;

  // wide form: stim, task (inputs) -> hidden -> response (BF16 edge)
  int n_inputs = 0;
  for (int i = 0; i < n_mech; ++i) n_inputs += mechs[i].kind == DG_INPUT;
  if (n_inputs == 2 && n_logistic == 2 && n_proj == 3 && n_ddm == 0) {
    int in0 = -1, in1 = -1, hid = -1, resp = stop->mech;
    for (int i = 0; i < n_mech; ++i) {
      if (mechs[i].kind == DG_INPUT) (in0 < 0 ? in0 : in1) = i;
      else if (i != resp) hid = i;
    }
    const dg_projection *ps = nullptr, *pt = nullptr, *pr = nullptr;
    for (int p = 0; p < n_proj; ++p) {
      if (projs[p].sender == in0 && projs[p].receiver == hid) ps = &projs[p];
      if (projs[p].sender == in1 && projs[p].receiver == hid) pt = &projs[p];
      if (projs[p].sender == hid && projs[p].receiver == resp) pr = &projs[p];
    }
    const int H = hid >= 0 ? mechs[hid].size : 0;
    const int nin = (in0 >= 0 ? mechs[in0].size : 0) + (in1 >= 0 ? mechs[in1].size : 0);
    if (ps && pt && pr && pr->dtype == DG_BF16 && H >= 64 && H <= 256 && H % 64 == 0 &&
        mechs[resp].size == 16 && dg::wide_smem_bytes(H, nin, true) <= 227 * 1024 &&
        dg::wide_smem_bytes(H, nin, false) <= 227 * 1024) {
      m->kind = K_WIDE;
      m->S = mechs[in0].size;
      m->T = mechs[in1].size;
      m->H = H;
      m->R = 16;
      m->bias_h = (float)mechs[hid].bias;
      m->gain_h = (float)mechs[hid].gain;
      m->bias_r = (float)mechs[resp].bias;
      m->gain_r = (float)mechs[resp].gain;
      // hidden weights: row h = [stimulus weights | task weights]
      const int S = m->S, T = m->T;
      std::vector<float> win((size_t)H * (S + T));
      for (int h = 0; h < H; ++h) {
        for (int j = 0; j < S; ++j) win[(size_t)h * (S + T) + j] = ps->weights[(size_t)h * S + j];
        for (int j = 0; j < T; ++j) win[(size_t)h * (S + T) + S + j] = pt->weights[(size_t)h * T + j];
      }
      std::vector<uint16_t> wr(16 * (size_t)H);
      std::vector<float> wrf(16 * (size_t)H);
      for (size_t i = 0; i < wr.size(); ++i) {
        wr[i] = to_bf16(pr->weights[i]);
        wrf[i] = from_bf16(wr[i]);
      }
      std::vector<uint16_t> img(16 * 2 * (size_t)H);
      dg::wide_b_image(wr.data(), H, img.data());
      dg_status st;
      if ((st = upload(&m->d_w_hid, win)) != DG_OK) return st;
      if ((st = upload(&m->d_w_resp_bf16, img)) != DG_OK) return st;
      if ((st = upload(&m->d_w_resp_f32, wrf)) != DG_OK) return st;
      m->n_inputs = S + T;
      return DG_OK;
    }
  }
  for (int p = 0; p < n_proj; ++p)
    if (projs[p].dtype != DG_F32)
      return fail(DG_E_UNSUPPORTED, "compose: BF16 weights only on the wide network's response edge");

  if (U > dg::kNetMaxUnits || n_in > dg::kNetMaxInputs)
    return fail(DG_E_UNSUPPORTED, "compose: small-network kernel takes <= %d logistic and <= %d input units",
                dg::kNetMaxUnits, dg::kNetMaxInputs);
  m->kind = K_NET;
  dg::NetLayout& L = m->layout;
  memset(&L, 0, sizeof L);
  L.U = U;
  L.n_in = n_in;
  L.rate = (float)rate;
  L.noise = (float)noise;
  L.stop_off = noff[stop->mech];
  L.stop_size = mechs[stop->mech].size;

  L.stop_threshold = (float)stop->threshold;
  L.max_steps = stop->max_steps;
  for (int i = 0; i < n_mech; ++i)
    if (noff[i] >= 0)
      for (int u = 0; u < mechs[i].size; ++u) {
        L.gain[noff[i] + u] = (float)mechs[i].gain;
        L.bias[noff[i] + u] = (float)mechs[i].bias;
      }
  std::vector<float> w_in((size_t)U * std::max(1, n_in), 0.f);
  std::vector<int> deg(U, 0);
  L.n_ddm = n_ddm;
  for (int i = 0; i < n_mech; ++i)
    if (doff[i] >= 0)
      for (int u = 0; u < mechs[i].size; ++u) {
        const int q = doff[i] + u;
        L.ddm_bias[q] = (float)mechs[i].bias;
        L.ddm_dt[q] = (float)mechs[i].dt;
        L.ddm_diffusion[q] = (float)(mechs[i].noise * std::sqrt(mechs[i].dt));
        L.ddm_z[q] = (float)mechs[i].threshold;
        L.ddm_max[q] = mechs[i].max_steps;
      }
  for (int p = 0; p < n_proj; ++p) {
    const auto& e = projs[p];
    const int rs = mechs[e.receiver].size, ss = mechs[e.sender].size;
    if (doff[e.receiver] >= 0) {  // into DDM nodes: weights over the stop layer's units
      for (int i = 0; i < rs; ++i)
        for (int j = 0; j < ss; ++j)
          L.ddm_w[doff[e.receiver] + i][j] += e.weights[(size_t)i * ss + j];
      continue;
    }
    for (int i = 0; i < rs; ++i)
      for (int j = 0; j < ss; ++j) {
        const float w = e.weights[(size_t)i * ss + j];
        const int dst = noff[e.receiver] + i;
        if (mechs[e.sender].kind == DG_INPUT) {
          w_in[(size_t)dst * n_in + ioff[e.sender] + j] += w;
        } else {
          if (deg[dst] >= dg::kNetMaxInDegree)
            return fail(DG_E_UNSUPPORTED,
                        "compose: a unit receives more than %d edges from logistic units",
                        dg::kNetMaxInDegree);
          L.src[dst][deg[dst]] = (int8_t)(noff[e.sender] + j);
          L.w[dst][deg[dst]] = w;
          ++deg[dst];
        }
      }
  }
  // each unit's incoming edges in sender order, one edge per sender (the
  // weights of repeated senders added): every form sums the same terms in the
  // same order, the one-lane form over a dense row of senders
  for (int u = 0; u < U; ++u) {
    std::vector<std::pair<int, double>> row;
    for (int d = 0; d < deg[u]; ++d) row.emplace_back((int)L.src[u][d], (double)L.w[u][d]);
    std::stable_sort(row.begin(), row.end(),
                     [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
                       return a.first < b.first;
                     });
    int n = 0;
    for (size_t i = 0; i < row.size(); ++i) {
      if (n > 0 && row[(size_t)n - 1].first == row[i].first)
        row[(size_t)n - 1].second += row[i].second;
      else
        row[(size_t)n++] = row[i];
    }
    for (int d = 0; d < dg::kNetMaxInDegree; ++d) {
      L.src[u][d] = d < n ? (int8_t)row[(size_t)d].first : (int8_t)0;
      L.w[u][d] = d < n ? (float)row[(size_t)d].second : 0.f;
    }
    deg[u] = n;
  }
  L.D = 0;
  for (int u = 0; u < U; ++u) L.D = std::max(L.D, deg[u]);
  dg_status st;
  if ((st = upload(&m->d_w_in, w_in)) != DG_OK) return st;
  DG_CUDA(cudaMalloc(&m->d_layout, sizeof(dg::NetLayout)));
  DG_CUDA(cudaMemcpy(m->d_layout, &L, sizeof L, cudaMemcpyHostToDevice));
  return DG_OK;
}

}  // namespace

namespace dg {

// Validate a grid search and fill its kernel parameters without touching any
// scratch or allocating anything; the caller supplies partials, ticket and,
// for the plain form without cand_means, the means buffer.
dg_status grid_params_noalloc(dg_model* m, const dg_grid_desc* d, dg_grid_result* result,
                              double* cand_means, GridParams* p) {
  dg_status st = check_grid_args(m, d, result);
  if (st != DG_OK) return st;
  *p = GridParams{};
  for (int i = 0; i < 3; ++i) {
    p->lv[i] = d->levels[i];
    p->L[i] = d->n_levels[i];
  }
  p->pos = d->positions;
  p->n_trials = d->n_trials;
  p->k0 = (uint32_t)d->seed;
  p->k1 = (uint32_t)(d->seed >> 32);
  p->rk = dg::philox_keys(p->k0, p->k1);
  p->offset = m->offset;
  p->weight = m->weight;
  const long long total = (long long)d->n_levels[0] * d->n_levels[1] * d->n_levels[2];
  p->cand0 = d->cand_begin;
  p->n_cand = d->cand_count ? d->cand_count : total;
  p->means = cand_means;
  p->result = result;
  return DG_OK;
}

dg_status set_error(dg_status s, const char* msg) { return fail(s, "%s", msg); }

int model_device(const dg_model* m) { return m->ctx->device; }

}  // namespace dg

// ===================================================================== ABI ===

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

const char* dg_version(void) { return "distill-gpu 0.1 sm_103a"; }

dg_status dg_create(dg_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return fail(DG_E_ARG, "dg_create: null out");
  int n = 0;
  DG_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(DG_E_ARG, "dg_create: device %d of %d", device, n);
  DG_CUDA(cudaSetDevice(device));
  DG_CUDA(cudaFree(nullptr));  // create the primary context
  dg_ctx* c = new dg_ctx;
  c->device = device;
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)150 * 1000 * 1000 * 1000;
  if (const char* e = getenv("DG_AUTOTUNE")) c->autotune = atoi(e) != 0;
  if (const char* e = getenv("DG_AUTOTUNE_CACHE")) c->tune_file = e;
  load_tune_file(c);
  *out = c;
  return DG_OK;
}

dg_status dg_destroy(dg_ctx* ctx) {
  if (!ctx) return fail(DG_E_ARG, "dg_destroy: null ctx");
  ctx->server.reset();
  // streams that own scratch may already be destroyed (serving slots, batch
  // branches): wait for the whole device instead of per stream
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->scratch) {
    cudaFree(kv.second.base);
    if (kv.second.means) cudaFree(kv.second.means);
    if (kv.second.ext) cudaFree(kv.second.ext);
    if (kv.second.perm) cudaFree(kv.second.perm);
    if (kv.second.net) cudaFree(kv.second.net);
    if (kv.second.gb) cudaFree(kv.second.gb);
  }
  delete ctx;
  return DG_OK;
}

dg_status dg_compose(dg_ctx* ctx, const dg_mechanism* mechs, int32_t n_mech,
                     const dg_projection* projs_in, int32_t n_proj, const dg_stop* stop,
                     uint64_t weight_seed, dg_model** out) {
  if (!ctx || !mechs || !stop || !out || n_mech < 1 || n_proj < 0 || (n_proj > 0 && !projs_in))
    return fail(DG_E_ARG, "dg_compose: null or empty arguments");
  // seeded weights: projection p, weight w: lo + (hi - lo) u in FP64, rounded
  // to FP32, u from word w & 3 of Philox(counter (p, 0, w >> 2, 2)) (Sec. 3.3
  // static parameters, drawn apart from all noise)
  std::vector<dg_projection> pj(projs_in, projs_in + n_proj);
  std::vector<std::vector<float>> pw(n_proj);
  for (int p = 0; p < n_proj; ++p) {
    dg_projection& q = pj[p];
    if (q.sender < 0 || q.sender >= n_mech || q.receiver < 0 || q.receiver >= n_mech)
      return fail(DG_E_SHAPE, "dg_compose: projection %d names a mechanism out of range", p);
    const size_t n = (size_t)mechs[q.receiver].size * (size_t)mechs[q.sender].size;
    if (!q.weights && (q.lo != 0.0 || q.hi != 0.0)) {
      if (!(q.lo < q.hi) || !std::isfinite(q.lo) || !std::isfinite(q.hi))
        return fail(DG_E_ARG, "dg_compose: projection %d: seeded weights need finite lo < hi", p);
      const uint32_t k0 = (uint32_t)weight_seed, k1 = (uint32_t)(weight_seed >> 32);
      pw[p].resize(n);
      for (size_t w = 0; w < n; w += 4) {
        const uint4 x = dg::philox(make_uint4((uint32_t)p, 0u, (uint32_t)(w >> 2), 2u), k0, k1);
        const uint32_t word[4] = {x.x, x.y, x.z, x.w};
        for (size_t i = 0; i < 4 && w + i < n; ++i) {
          const double u = ((double)(word[i] >> 9) + 0.5) * 0x1p-23;
          const double span = q.hi - q.lo;
          const double scaled = span * u;    // host code is built without contraction
          pw[p][w + i] = (float)(q.lo + scaled);
        }
      }
      q.weights = pw[p].data();
    } else if (q.weights) {
      pw[p].assign(q.weights, q.weights + n);
    }
  }
  const dg_projection* projs = n_proj ? pj.data() : nullptr;
  if (stop->max_steps < 1) return fail(DG_E_ARG, "dg_compose: stop.max_steps must be >= 1");
  for (int i = 0; i < n_mech; ++i) {
    if (mechs[i].kind < DG_INPUT || mechs[i].kind > DG_PP_OBJECTIVE)
      return fail(DG_E_ARG, "dg_compose: mechanism %d has unknown kind %d", i, mechs[i].kind);
    if (mechs[i].size < 1) return fail(DG_E_SHAPE, "dg_compose: mechanism %d has size < 1", i);
  }
  DG_CUDA(cudaSetDevice(ctx->device));
  std::unique_ptr<dg_model> m(new dg_model);
  m->ctx = ctx;
  m->proj_w = std::move(pw);
  int counts[7] = {0};
  for (int i = 0; i < n_mech; ++i) counts[mechs[i].kind]++;
  const int integrators = counts[DG_DDM] + counts[DG_LCA];
  const int pp = counts[DG_PP_OBSERVE] + counts[DG_PP_ACTION] + counts[DG_PP_OBJECTIVE];

  if (integrators > 0 && counts[DG_TRANSFER_LOGISTIC] == 0) {
    if (integrators != 1 || pp || counts[DG_INPUT] > 1)
      return fail(DG_E_SHAPE, "dg_compose: an integrator model has one DDM or LCA (and at most one input)");
    int im = -1, in = -1;
    for (int i = 0; i < n_mech; ++i) {
      if (mechs[i].kind == DG_DDM || mechs[i].kind == DG_LCA) im = i;
      else in = i;
    }
    const dg_mechanism& g = mechs[im];
    if (in >= 0) {
      if (mechs[in].size != g.size)
        return fail(DG_E_SHAPE, "dg_compose: input size %d != integrator size %d", mechs[in].size, g.size);
      if (n_proj != 1 || projs[0].sender != in || projs[0].receiver != im || projs[0].weights)
        return fail(DG_E_SHAPE, "dg_compose: input feeds the integrator by one identity projection (NULL weights)");
    } else if (n_proj != 0) {
      return fail(DG_E_SHAPE, "dg_compose: integrator model without input takes no projections");
    }
    if (stop->mech != im) return fail(DG_E_SHAPE, "dg_compose: stop must name the integrator");
    if (!(g.dt > 0.0) || !(g.noise >= 0.0))
      return fail(DG_E_ARG, "dg_compose: integrator needs dt > 0 and noise >= 0");
    m->dt = (float)g.dt;
    m->sigma = (float)g.noise;
    m->diffusion = (float)(g.noise * std::sqrt(g.dt));
    m->max_steps = stop->max_steps;
    if (g.kind == DG_DDM) {
      if (g.size != 1) return fail(DG_E_SHAPE, "dg_compose: DDM has size 1");
      m->kind = K_DDM;
      m->x0 = (float)g.start;
      m->state_size = 1;
    } else {
      if (g.size > 16) return fail(DG_E_UNSUPPORTED, "dg_compose: LCA size %d > 16", g.size);
      if ((g.flags & DG_LCA_TWO_SIDED) && g.size != 1)
        return fail(DG_E_SHAPE, "dg_compose: two-sided LCA needs size 1");
      if (!(stop->threshold > 0.0)) return fail(DG_E_ARG, "dg_compose: LCA threshold must be > 0");
      m->kind = K_LCA;
      m->N = g.size;
      m->leak = (float)g.leak;
      m->inhibition = (float)g.inhibition;
      m->threshold = (float)stop->threshold;
      m->rectify = (g.flags & DG_LCA_NO_RECTIFY) ? 0 : 1;
      m->two_sided = (g.flags & DG_LCA_TWO_SIDED) ? 1 : 0;
      m->state_size = g.size;
    }
    *out = m.release();
    return DG_OK;
  }

  if (pp > 0) {
    if (n_mech != 4 || counts[DG_INPUT] != 1 || counts[DG_PP_OBSERVE] != 1 ||
        counts[DG_PP_ACTION] != 1 || counts[DG_PP_OBJECTIVE] != 1)
      return fail(DG_E_SHAPE, "dg_compose: predator-prey model is input -> observe -> action -> objective");
    int idx[7] = {-1, -1, -1, -1, -1, -1, -1};
    for (int i = 0; i < n_mech; ++i) idx[mechs[i].kind] = i;
    if (mechs[idx[DG_INPUT]].size != 6 || mechs[idx[DG_PP_OBSERVE]].size != 6 ||
        mechs[idx[DG_PP_ACTION]].size != 2 || mechs[idx[DG_PP_OBJECTIVE]].size != 1)
      return fail(DG_E_SHAPE, "dg_compose: predator-prey sizes are 6, 6, 2, 1");
    const int chain[4] = {idx[DG_INPUT], idx[DG_PP_OBSERVE], idx[DG_PP_ACTION], idx[DG_PP_OBJECTIVE]};
    if (n_proj != 3) return fail(DG_E_SHAPE, "dg_compose: predator-prey model has 3 projections");
    for (int k = 0; k < 3; ++k) {
      bool found = false;
      for (int p = 0; p < n_proj; ++p)
        if (projs[p].sender == chain[k] && projs[p].receiver == chain[k + 1] && !projs[p].weights)
          found = true;
      if (!found) return fail(DG_E_SHAPE, "dg_compose: predator-prey projection %d -> %d missing", chain[k], chain[k + 1]);
    }
    const double off = mechs[idx[DG_PP_OBSERVE]].offset;
    if (!(off > 0.0)) return fail(DG_E_ARG, "dg_compose: observation offset must be > 0");
    m->kind = K_PP;
    m->offset = (float)off;
    m->weight = (float)mechs[idx[DG_PP_ACTION]].weight;
    m->offset_d = off;
    m->weight_d = mechs[idx[DG_PP_ACTION]].weight;
    m->max_steps = stop->max_steps;
    *out = m.release();
    return DG_OK;
  }

  dg_status st = compose_transfer(m.get(), mechs, n_mech, projs, n_proj, stop);
  if (st != DG_OK) {
    dg_model_free(m.release());
    return st;
  }
  // the weight copies (from pageable memory) must have landed before any
  // stream, blocking or not, launches on this model
  DG_CUDA(cudaDeviceSynchronize());
  *out = m.release();
  return DG_OK;
}

dg_status dg_model_free(dg_model* m) {
  if (!m) return fail(DG_E_ARG, "dg_model_free: null model");
  cudaFree(m->d_layout);
  cudaFree(m->d_w_in);
  cudaFree(m->d_w_hid);
  cudaFree(m->d_w_resp_bf16);
  cudaFree(m->d_w_resp_f32);
  delete m;
  return DG_OK;
}

dg_status dg_model_weights(const dg_model* m, int32_t proj, float* out, int64_t n) {
  if (!m || proj < 0 || proj >= (int32_t)m->proj_w.size())
    return fail(DG_E_ARG, "dg_model_weights: projection out of range");
  const auto& w = m->proj_w[proj];
  if (n != (int64_t)w.size())
    return fail(DG_E_ARG, "dg_model_weights: projection %d holds %lld weights, not %lld", proj,
                (long long)w.size(), (long long)n);
  if (n > 0 && !out) return fail(DG_E_ARG, "dg_model_weights: null output");
  if (n > 0) memcpy(out, w.data(), (size_t)n * sizeof(float));
  return DG_OK;
}

dg_status dg_model_info(const dg_model* m, int32_t* kind, int32_t* state_size) {
  if (!m) return fail(DG_E_ARG, "dg_model_info: null model");
  if (kind) *kind = m->kind;
  if (state_size) *state_size = m->state_size;
  return DG_OK;
}

dg_status dg_run(dg_model* m, const dg_run_desc* d, int8_t* choice, int32_t* step,
                 float* final_state, void* stream) {
  dg_status st = check_run_args(m, d, choice, step);
  if (st != DG_OK) return st;
  DG_CUDA(cudaSetDevice(m->ctx->device));
  return run_device(m, d, choice, step, final_state, (cudaStream_t)stream);
}

dg_status dg_run_jobs(dg_model* m, int32_t n_jobs, const dg_run_desc* descs,
                      int8_t* const* choice, int32_t* const* step, float* const* final_state,
                      void* stream) {
  dg_status st = check_jobs_args(m, n_jobs, descs, choice, step);
  if (st != DG_OK) return st;
  DG_CUDA(cudaSetDevice(m->ctx->device));
  return run_jobs_device(m, n_jobs, descs, choice, step, final_state, (cudaStream_t)stream);
}

dg_status dg_grid_search(dg_model* m, const dg_grid_desc* d, dg_grid_result* result,
                         double* cand_means, void* stream) {
  dg_status st = check_grid_args(m, d, result);
  if (st != DG_OK) return st;
  DG_CUDA(cudaSetDevice(m->ctx->device));
  return grid_device(m, d, result, cand_means, (cudaStream_t)stream);
}

dg_status dg_grid_search_batch(dg_model* m, int32_t n_searches, const dg_grid_desc* descs,
                               dg_grid_result* results, double* const* cand_means, void* stream) {
  dg_status st = check_grid_batch(m, n_searches, descs, results);
  if (st != DG_OK) return st;
  DG_CUDA(cudaSetDevice(m->ctx->device));
  std::vector<dg_grid_result*> res((size_t)n_searches);
  for (int i = 0; i < n_searches; ++i) res[(size_t)i] = results + i;
  return grid_batch_device(m, n_searches, descs, res.data(), cand_means, (cudaStream_t)stream);
}

dg_status dg_argmax_f64(dg_ctx* ctx, const double* values, int64_t n, dg_grid_result* result,
                        void* stream) {
  if (!ctx || !values || !result || n < 1) return fail(DG_E_ARG, "dg_argmax_f64: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch* sc = nullptr;
  dg_status st = get_scratch(ctx, s, &sc);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemsetAsync(sc->ticket(), 0, 4, s));
  DG_CUDA(dg::launch_argmax(values, n, sc->partials(), sc->ticket(), result, s));
  return DG_OK;
}

dg_status dg_run_episodes(dg_model* m, const dg_episode_desc* d, const dg_episode_out* o,
                          void* stream) {
  if (!m || !d || !o || !o->outcome || !o->steps)
    return fail(DG_E_ARG, "dg_run_episodes: null model, desc or outputs");
  if (m->kind != K_PP)
    return fail(DG_E_UNSUPPORTED, "dg_run_episodes: model is not a predator-prey model");
  if (d->n_episodes < 1) return fail(DG_E_ARG, "dg_run_episodes: n_episodes must be >= 1");
  if (d->n_trials < 1 || d->n_trials > 1024)
    return fail(DG_E_ARG, "dg_run_episodes: n_trials %d out of [1, 1024]", d->n_trials);
  if (d->max_steps < 1 || (long long)d->max_steps * d->n_trials > (1ll << 32))
    return fail(DG_E_ARG, "dg_run_episodes: max_steps must be >= 1 with max_steps n_trials <= 2^32");
  for (int i = 0; i < 3; ++i) {
    if (d->n_levels[i] < 1 || d->n_levels[i] > 4096 || !d->levels[i])
      return fail(DG_E_ARG, "dg_run_episodes: levels of signal %d", i);
    if (!(d->speed[i] >= 0.0) || !std::isfinite(d->speed[i]))
      return fail(DG_E_ARG, "dg_run_episodes: speed %d must be finite and >= 0", i);
  }
  if (!(d->capture_radius >= 0.0) || !std::isfinite(d->capture_radius))
    return fail(DG_E_ARG, "dg_run_episodes: capture_radius must be finite and >= 0");
  if (!d->start) return fail(DG_E_ARG, "dg_run_episodes: null start positions");
  if (d->episode_offset < 0 || d->episode_offset + d->n_episodes > INT32_MAX)
    return fail(DG_E_ARG, "dg_run_episodes: episode_offset + n_episodes must lie in [0, 2^31 - 1]");
  const long long n_cand = (long long)d->n_levels[0] * d->n_levels[1] * d->n_levels[2];
  if (n_cand > 0xFFFFFFFFll) return fail(DG_E_ARG, "dg_run_episodes: more than 2^32 - 1 candidates");
  const long long cpe = (n_cand + dg::kEpisodeChunk - 1) / dg::kEpisodeChunk;
  const long long E = d->n_episodes;
  if (E * cpe > (1ll << 40)) return fail(DG_E_ARG, "dg_run_episodes: too much work per step");
  if (E > (1ll << 30)) return fail(DG_E_ARG, "dg_run_episodes: too many episodes");
  DG_CUDA(cudaSetDevice(m->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Scratch* sc = nullptr;
  dg_status st = get_scratch(m->ctx, s, &sc);
  if (st != DG_OK) return st;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t b_state = up(sizeof(float) * 6 * E), b_active = up(sizeof(int) * 3 * E),
               b_count = 256, b_ticket = up(sizeof(unsigned) * E),
               b_part = up(sizeof(dg::TopTwo) * (size_t)(E * cpe));
  st = scratch_ext(m->ctx, sc, b_state + b_active + b_count + b_ticket + b_part, s);
  if (st != DG_OK) return st;
  unsigned char* x = sc->ext;
  dg::EpisodeParams p{};
  for (int i = 0; i < 3; ++i) {
    p.lv[i] = d->levels[i];
    p.L[i] = d->n_levels[i];
    p.speed[i] = d->speed[i];
  }
  p.n_cand = n_cand;
  p.cpe = (int)cpe;
  p.n_trials = d->n_trials;
  p.k0 = (uint32_t)d->seed;
  p.k1 = (uint32_t)(d->seed >> 32);
  p.rk = dg::philox_keys(p.k0, p.k1);
  p.offset = m->offset;
  p.weight = m->weight;
  p.offset_d = m->offset_d;
  p.weight_d = m->weight_d;
  p.radius = d->capture_radius;
  p.E = (int)E;
  p.T = d->max_steps;
  p.e0 = (uint32_t)d->episode_offset;
  p.start = d->start;
  p.state = reinterpret_cast<float*>(x);
  p.active = reinterpret_cast<int*>(x + b_state);
  p.count = reinterpret_cast<int*>(x + b_state + b_active);
  p.cursor = reinterpret_cast<unsigned long long*>(x + b_state + b_active + 64);
  p.ticket = reinterpret_cast<unsigned int*>(x + b_state + b_active + b_count);
  p.partials = reinterpret_cast<dg::TopTwo*>(x + b_state + b_active + b_count + b_ticket);
  p.outcome = o->outcome;
  p.steps = o->steps;
  p.final_pos = o->final_pos;
  p.traj_best = o->best;
  p.traj_value = o->value;
  p.traj_pos = o->pos;
  DG_CUDA(dg::launch_episode_init(p, s));
  for (int t = 0; t < p.T; ++t) {
    p.t = t;
    DG_CUDA(dg::launch_episode_step(p, s));
  }
  return DG_OK;
}

dg_status dg_grid_refine(dg_model* m, const dg_refine_desc* d, dg_refine_round* rounds,
                         void* stream) {
  if (!m || !d || !rounds) return fail(DG_E_ARG, "dg_grid_refine: null model, desc or rounds");
  if (m->kind != K_PP)
    return fail(DG_E_UNSUPPORTED, "dg_grid_refine: model is not a predator-prey model");
  const int G = d->points, R = d->rounds;
  if (G < 4 || G > dg::kRefineMaxPoints)
    return fail(DG_E_ARG, "dg_grid_refine: points %d out of [4, %d]", G, dg::kRefineMaxPoints);
  const long long n_cand = (long long)G * G * G;
  if (R < 1 || (long long)R * n_cand > (1ll << 32))
    return fail(DG_E_ARG, "dg_grid_refine: rounds %d out of [1, 2^32 / points^3]", R);
  if (d->n_trials < 1 || d->n_trials > 1024)
    return fail(DG_E_ARG, "dg_grid_refine: n_trials %d out of [1, 1024]", d->n_trials);
  if (!d->positions) return fail(DG_E_ARG, "dg_grid_refine: null positions");
  for (int e = 0; e < 3; ++e)
    if (!std::isfinite(d->lo[e]) || !std::isfinite(d->hi[e]) || !(d->lo[e] <= d->hi[e]))
      return fail(DG_E_ARG, "dg_grid_refine: domain of signal %d is not a finite lo <= hi", e);
  DG_CUDA(cudaSetDevice(m->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  // up to 8,192 candidates a round: the whole search as one cluster launch
  // (DG_REFINE_FUSED=0 selects the launch-per-round form)
  const char* fe = getenv("DG_REFINE_FUSED");
  if (n_cand <= 8192 && !(fe && atoi(fe) == 0)) {
    dg::RefineFusedParams fp{};
    for (int e = 0; e < 3; ++e) {
      fp.lo0[e] = d->lo[e];
      fp.hi0[e] = d->hi[e];
    }
    fp.G = G;
    fp.R = R;
    fp.n_trials = d->n_trials;
    fp.pos = d->positions;
    fp.rk = dg::philox_keys((uint32_t)d->seed, (uint32_t)(d->seed >> 32));
    fp.offset = m->offset;
    fp.weight = m->weight;
    fp.rounds = rounds;
    DG_CUDA(dg::launch_refine_fused(fp, s));
    return DG_OK;
  }
  Scratch* sc = nullptr;
  dg_status st = get_scratch(m->ctx, s, &sc);
  if (st != DG_OK) return st;
  dg::RefineParams rp{};
  for (int e = 0; e < 3; ++e) {
    rp.lo0[e] = d->lo[e];
    rp.hi0[e] = d->hi[e];
  }
  rp.G = G;
  rp.R = R;
  rp.lv = sc->refine_levels();
  rp.rounds = rounds;
  rp.ticket = sc->ticket();
  dg::GridParams p{};
  p.pos = d->positions;
  p.n_trials = d->n_trials;
  p.k0 = (uint32_t)d->seed;
  p.k1 = (uint32_t)(d->seed >> 32);
  p.rk = dg::philox_keys(p.k0, p.k1);
  p.offset = m->offset;
  p.weight = m->weight;
  p.cand0 = 0;
  p.n_cand = n_cand;
  p.partials = sc->partials();
  p.ticket = sc->ticket();
  for (int e = 0; e < 3; ++e) p.L[e] = G;
  DG_CUDA(dg::launch_refine_init(rp, s));
  for (int r = 0; r < R; ++r) {
    for (int e = 0; e < 3; ++e) p.lv[e] = rp.lv + ((r & 1) * 3 + e) * dg::kRefineMaxPoints;
    p.stream0 = (uint32_t)((long long)r * n_cand);
    // the round's dg_grid_result fields (best_index, value, gap) sit at byte 40
    p.result = reinterpret_cast<unsigned char*>(rounds + r) + offsetof(dg_refine_round, best_index);
    DG_CUDA(dg::launch_grid(p, DG_MODE_BATCHED, dg::LaunchCfg{}, s));
    DG_CUDA(dg::launch_refine_step(rp, r, s));
  }
  return DG_OK;
}

dg_status dg_argmax_f64_reservoir(dg_ctx* ctx, const double* values, int64_t n, uint64_t seed,
                                  dg_grid_result* result, void* stream) {
  if (!ctx || !values || !result || n < 1)
    return fail(DG_E_ARG, "dg_argmax_f64_reservoir: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch* sc = nullptr;
  dg_status st = get_scratch(ctx, s, &sc);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemsetAsync(sc->ticket(), 0, 4, s));
  DG_CUDA(dg::launch_argmax(values, n, sc->partials(), sc->ticket(), result, s));
  DG_CUDA(dg::launch_tie_reservoir(values, n, 0, seed, result, s));
  return DG_OK;
}

dg_status dg_stream_status(dg_ctx* ctx, void* stream) {
  if (!ctx) return fail(DG_E_ARG, "dg_stream_status: null ctx");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(ctx->device));
  DG_CUDA(cudaStreamSynchronize(s));
  Scratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->scratch.find(s);
    if (it == ctx->scratch.end()) return DG_OK;  // nothing ran on this stream
    sc = &it->second;
  }
  int word = 0;
  DG_CUDA(cudaMemcpyAsync(&word, sc->status(), sizeof word, cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (word == 0) return DG_OK;
  DG_CUDA(cudaMemsetAsync(sc->status(), 0, sizeof word, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return fail(DG_E_TIMEOUT, "a device-side wait gave up (status %d); affected outputs unwritten",
              word);
}

dg_status dg_selftest_wait_timeout(dg_ctx* ctx, int32_t wait_us, void* stream) {
  if (!ctx || wait_us < 1 || wait_us > 2000000)
    return fail(DG_E_ARG, "dg_selftest_wait_timeout: wait_us must be in [1, 2e6]");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(ctx->device));
  Scratch* sc = nullptr;
  dg_status st = get_scratch(ctx, s, &sc);
  if (st != DG_OK) return st;
  int khz = 0;
  DG_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
  if (khz <= 0) khz = 2000000;
  DG_CUDA(dg::launch_wait_timeout((long long)wait_us * khz / 1000, sc->status(), s));
  return DG_OK;
}

dg_status dg_selftest_pair_sum(const float* values, int64_t n_groups, int32_t per_group,
                               int32_t lanes, double* means, void* stream) {
  if (n_groups < 0 || per_group < 1 || per_group > 1024 || (lanes != 8 && lanes != 32) ||
      (n_groups > 0 && (!values || !means)))
    return fail(DG_E_ARG,
                "dg_selftest_pair_sum: need n_groups >= 0, per_group in [1, 1024], lanes 8 or 32, "
                "non-null pointers");
  if (n_groups > (int64_t)1 << 40)
    return fail(DG_E_ARG, "dg_selftest_pair_sum: n_groups too large");
  DG_CUDA(dg::launch_pair_sum(values, n_groups, per_group, lanes, means, (cudaStream_t)stream));
  return DG_OK;
}

dg_status dg_philox_words(uint64_t seed, uint32_t trial, uint32_t cand, uint32_t purpose,
                          uint32_t block0, int64_t nblocks, uint32_t* out, void* stream) {
  if (nblocks < 0 || (nblocks > 0 && !out)) return fail(DG_E_ARG, "dg_philox_words: bad arguments");
  if (((uintptr_t)out & 15u) != 0) return fail(DG_E_ARG, "dg_philox_words: out must be 16-byte aligned");
  DG_CUDA(dg::launch_philox_words(seed, trial, cand, purpose, block0, nblocks, out,
                                  (cudaStream_t)stream));
  return DG_OK;
}

dg_status dg_normals(uint64_t seed, uint32_t trial, uint32_t cand, uint64_t d0, int64_t n,
                     float* out, void* stream) {
  if (n < 0 || (n > 0 && !out)) return fail(DG_E_ARG, "dg_normals: bad arguments");
  DG_CUDA(dg::launch_normals(seed, trial, cand, d0, n, out, (cudaStream_t)stream));
  return DG_OK;
}

// ---------------------------------------------------------------- batch ---

struct dg_batch {
  dg_ctx* ctx;
  struct Op {
    dg_model* m;
    bool grid;
    dg_run_desc run;
    dg_grid_desc gd;
    int8_t* choice;
    int32_t* step;
    float* fs;
    dg_grid_result* res;
    double* means;
  };
  std::vector<Op> ops;
  std::vector<cudaStream_t> side;
  cudaStream_t cap = nullptr;  // private capture stream (the legacy stream cannot be captured)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;         // kernel nodes of the captured graph
};

dg_status dg_batch_create(dg_ctx* ctx, dg_batch** out) {
  if (!ctx || !out) return fail(DG_E_ARG, "dg_batch_create: null argument");
  dg_batch* b = new dg_batch;
  b->ctx = ctx;
  *out = b;
  return DG_OK;
}

dg_status dg_batch_add_run(dg_batch* b, dg_model* m, const dg_run_desc* d, int8_t* choice,
                           int32_t* step, float* final_state) {
  if (!b) return fail(DG_E_ARG, "dg_batch_add_run: null batch");
  if (b->exec) return fail(DG_E_STATE, "dg_batch_add_run: batch already launched");
  dg_status st = check_run_args(m, d, choice, step);
  if (st != DG_OK) return st;
  dg_batch::Op op{};
  op.m = m;
  op.grid = false;
  op.run = *d;
  op.choice = choice;
  op.step = step;
  op.fs = final_state;
  b->ops.push_back(op);
  return DG_OK;
}

dg_status dg_batch_add_grid(dg_batch* b, dg_model* m, const dg_grid_desc* d,
                            dg_grid_result* result, double* cand_means) {
  if (!b) return fail(DG_E_ARG, "dg_batch_add_grid: null batch");
  if (b->exec) return fail(DG_E_STATE, "dg_batch_add_grid: batch already launched");
  dg_status st = check_grid_args(m, d, result);
  if (st != DG_OK) return st;
  dg_batch::Op op{};
  op.m = m;
  op.grid = true;
  op.gd = *d;
  op.res = result;
  op.means = cand_means;
  b->ops.push_back(op);
  return DG_OK;
}

static dg_status batch_op(dg_batch::Op& op, cudaStream_t s) {
  if (op.grid) return grid_device(op.m, &op.gd, op.res, op.means, s);
  return run_device(op.m, &op.run, op.choice, op.step, op.fs, s);
}

dg_status dg_batch_launch(dg_batch* b, void* stream) {
  if (!b) return fail(DG_E_ARG, "dg_batch_launch: null batch");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(b->ctx->device));
  if (b->exec) {
    DG_CUDA(cudaGraphLaunch(b->exec, s));
    return DG_OK;
  }
  if (b->ops.empty()) return DG_OK;
  // one forked stream per op; scratch and tuned shapes prepared outside capture
  for (size_t i = 0; i < b->ops.size(); ++i) {
    cudaStream_t side;
    DG_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    b->side.push_back(side);
    cudaEvent_t e;
    DG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->join.push_back(e);
    dg_status st = batch_op(b->ops[i], side);  // tunes shapes, allocates scratch
    if (st != DG_OK) return st;
  }
  for (auto side : b->side) DG_CUDA(cudaStreamSynchronize(side));
  DG_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  DG_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  cudaStream_t cs = b->cap;
  DG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  dg_status st = DG_OK;
  if (cudaEventRecord(b->fork, cs) != cudaSuccess) st = fail(DG_E_CUDA, "batch: fork record");
  for (size_t i = 0; i < b->ops.size() && st == DG_OK; ++i) {
    if (cudaStreamWaitEvent(b->side[i], b->fork, 0) != cudaSuccess) {
      st = fail(DG_E_CUDA, "batch: fork wait");
      break;
    }
    st = batch_op(b->ops[i], b->side[i]);
    if (st != DG_OK) break;
    if (cudaEventRecord(b->join[i], b->side[i]) != cudaSuccess ||
        cudaStreamWaitEvent(cs, b->join[i], 0) != cudaSuccess)
      st = fail(DG_E_CUDA, "batch: join");
  }
  cudaGraph_t g = nullptr;
  cudaError_t ec = cudaStreamEndCapture(cs, &g);
  if (st != DG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ec != cudaSuccess) return fail(DG_E_CUDA, "batch: end capture: %s", cudaGetErrorString(ec));
  {
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++b->kernels;
        }
    }
  }
  ec = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (ec != cudaSuccess) return fail(DG_E_CUDA, "batch: instantiate: %s", cudaGetErrorString(ec));
  DG_CUDA(cudaGraphLaunch(b->exec, s));
  return DG_OK;
}

dg_status dg_batch_kernels(const dg_batch* b, int64_t* n_kernels) {
  if (!b || !n_kernels) return fail(DG_E_ARG, "dg_batch_kernels: null argument");
  if (!b->exec) return fail(DG_E_STATE, "dg_batch_kernels: batch not launched yet");
  *n_kernels = b->kernels;
  return DG_OK;
}

dg_status dg_batch_free(dg_batch* b) {
  if (!b) return fail(DG_E_ARG, "dg_batch_free: null batch");
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->side) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return DG_OK;
}

// -------------------------------------------------------------- serving ---

dg_status dg_submit(dg_ctx* ctx, const dg_job* job, uint64_t* ticket) {
  if (!ctx || !job || !ticket || !job->model) return fail(DG_E_ARG, "dg_submit: null argument");
  dg_status st;
  if (job->is_grid) {
    if (!job->grid_result) return fail(DG_E_ARG, "dg_submit: grid job needs grid_result");
    st = check_grid_args(job->model, &job->grid, job->grid_result);
  } else {
    st = check_run_args(job->model, &job->run, job->choice, job->step);
  }
  if (st != DG_OK) return st;
  Server* sv = server_of(ctx);
  auto r = std::make_shared<JobRec>();
  r->job = *job;
  r->bytes = Server::job_bytes(*job);
  if (r->bytes > ctx->budget)
    return fail(DG_E_BUDGET, "dg_submit: job needs %zu bytes, budget is %zu", r->bytes, ctx->budget);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(sv->mu);
    r->id = sv->next_id++;
    sv->jobs[r->id] = r;
    sv->queue.push_back(r->id);
  }
  sv->cv_work.notify_all();
  *ticket = r->id;
  return DG_OK;
}

dg_status dg_wait(dg_ctx* ctx, uint64_t ticket, int32_t timeout_ms, dg_job_result* result) {
  if (!ctx) return fail(DG_E_ARG, "dg_wait: null ctx");
  Server* sv = server_of(ctx);
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return fail(DG_E_ARG, "dg_wait: unknown ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<JobRec> r = it->second;
  auto done = [&] { return r->state == 2; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, done);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return fail(DG_E_TIMEOUT, "dg_wait: ticket %llu not done after %d ms",
                (unsigned long long)ticket, timeout_ms);
  }
  if (result) {
    result->status = r->status;
    result->t_submit = r->t_submit;
    result->t_admit = r->t_admit;
    result->t_done = r->t_done;
    result->device_bytes = r->bytes;
  }
  sv->jobs.erase(ticket);
  if (r->status != DG_OK) return fail((dg_status)r->status, "job %llu failed", (unsigned long long)ticket);
  return DG_OK;
}

dg_status dg_tune_stats(dg_ctx* ctx, int64_t* tuned_keys, int64_t* untuned_launches) {
  if (!ctx) return fail(DG_E_ARG, "dg_tune_stats: null ctx");
  if (tuned_keys) {
    std::lock_guard<std::mutex> g(ctx->mu);
    *tuned_keys = (int64_t)ctx->tuned.size();
  }
  if (untuned_launches) *untuned_launches = ctx->untuned.load();
  return DG_OK;
}

dg_status dg_serve_stats(dg_ctx* ctx, int64_t* queued, int64_t* running, int64_t* done,
                         uint64_t* bytes_in_use) {
  if (!ctx) return fail(DG_E_ARG, "dg_serve_stats: null ctx");
  Server* sv = server_of(ctx);
  std::lock_guard<std::mutex> g(sv->mu);
  if (queued) *queued = (int64_t)sv->queue.size();
  if (running) *running = sv->n_running;
  if (done) *done = sv->n_done;
  if (bytes_in_use) *bytes_in_use = sv->in_use;
  return DG_OK;
}

}  // extern "C"
