// dg_grid_search_noalloc: the predator-prey grid search without any device
// memory allocation. dg_grid_search takes its scratch (the last-block argmax
// ticket, one argmax partial per block, and for the plain form a per-candidate
// means buffer) from memory the library allocates on first use of a stream.
// This entry point instead uses one fixed array in the library's own device
// memory, so it never calls an allocator.
#include <cuda_runtime.h>

#include <mutex>

#include "distill_gpu.h"
#include "dg_internal.h"

namespace dg {
dg_status grid_params_noalloc(dg_model* m, const dg_grid_desc* d, dg_grid_result* result,
                              double* cand_means, GridParams* p);
dg_status set_error(dg_status s, const char* msg);
int model_device(const dg_model* m);
}  // namespace dg

namespace {

constexpr int kBlocks = 1024;                 // argmax partials: one per block
constexpr long long kMaxCandidates = 32768;   // plain form without cand_means
constexpr size_t kHeader = 256;               // ticket
constexpr size_t kPartialsBytes = kBlocks * sizeof(dg::TopTwo);      // 24 KiB
constexpr size_t kMeansBytes = kMaxCandidates * sizeof(double);      // 256 KiB
constexpr size_t kScratchBytes = kHeader + kPartialsBytes + kMeansBytes;
constexpr int kMaxDevices = 64;

// Loaded with the library on every GPU that uses it and held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `dev` (which must be current). In
// host code the array's name is only a host-side stand-in, so the address is
// looked up once per device and cached.
dg_status scratch_on(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices)
    return dg::set_error(DG_E_UNSUPPORTED, "dg_grid_search_noalloc: device index >= 64");
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return dg::set_error(DG_E_CUDA, "dg_grid_search_noalloc: cudaGetSymbolAddress failed");
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_grid_search_noalloc(dg_model* model, const dg_grid_desc* desc,
                                            dg_grid_result* result, double* cand_means,
                                            void* stream) {
  dg::GridParams p;
  dg_status st = dg::grid_params_noalloc(model, desc, result, cand_means, &p);
  if (st != DG_OK) return st;
  const bool plain = desc->mode == DG_MODE_PLAIN;
  const bool reservoir = desc->tie_break == DG_TIE_RESERVOIR;
  const bool need_means = (plain || reservoir) && !cand_means;
  if (need_means && p.n_cand > kMaxCandidates)
    return dg::set_error(DG_E_ARG,
                         "dg_grid_search_noalloc: the plain form or the reservoir tie-break "
                         "without cand_means holds at most 32768 candidate means in its fixed "
                         "scratch; pass cand_means or evaluate fewer candidates per call");
  const int dev = dg::model_device(model);
  if (cudaSetDevice(dev) != cudaSuccess)
    return dg::set_error(DG_E_CUDA, "dg_grid_search_noalloc: cudaSetDevice failed");
  unsigned char* base = nullptr;
  st = scratch_on(dev, &base);
  if (st != DG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p.ticket = reinterpret_cast<unsigned int*>(base);
  p.partials = reinterpret_cast<dg::TopTwo*>(base + kHeader);
  if (need_means) p.means = reinterpret_cast<double*>(base + kHeader + kPartialsBytes);
  // the array keeps the previous call's contents: the ticket must start at 0
  if (cudaMemsetAsync(p.ticket, 0, sizeof(unsigned int), s) != cudaSuccess)
    return dg::set_error(DG_E_CUDA, "dg_grid_search_noalloc: ticket reset failed");
  dg::LaunchCfg cfg;
  cfg.block = 256;
  const int want = dg::grid_blocks(0, p.n_cand, p.n_trials, dg::grid_lanes(p.L));
  cfg.grid = want < kBlocks ? want : kBlocks;
  if (cfg.grid < 1) cfg.grid = 1;
  cudaError_t e = dg::launch_grid(p, plain ? 1 : 0, cfg, s);
  if (e == cudaSuccess && reservoir)
    e = dg::launch_tie_reservoir(p.means, p.n_cand, p.cand0, desc->seed, result, s);
  if (e != cudaSuccess) return dg::set_error(DG_E_CUDA, cudaGetErrorString(e));
  return DG_OK;
}
