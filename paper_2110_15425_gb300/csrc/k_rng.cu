// Replay of the kernels' random streams, so tests can compare raw Philox
// words bit for bit and normals within rounding against an independent
// implementation. Uses the same device functions as every model kernel.
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

namespace {

__global__ void philox_words_kernel(uint32_t k0, uint32_t k1, uint32_t trial, uint32_t cand,
                                    uint32_t purpose, uint32_t block0, long long nblocks,
                                    uint4* out) {
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblocks;
       b += (long long)gridDim.x * blockDim.x)
    out[b] = philox(make_uint4(trial, cand, block0 + (uint32_t)b, purpose), k0, k1);
}

__global__ void normals_kernel(uint32_t k0, uint32_t k1, uint32_t trial, uint32_t cand,
                               unsigned long long d0, long long n, float* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long d = d0 + (unsigned long long)i;
    const float4 z = normals4(noise_block(k0, k1, trial, cand, (uint32_t)(d >> 2)));
    out[i] = pick4(z, (uint32_t)(d & 3ull));
  }
}

}  // namespace

cudaError_t launch_philox_words(uint64_t seed, uint32_t trial, uint32_t cand, uint32_t purpose,
                                uint32_t block0, int64_t nblocks, uint32_t* out, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  long long g = (nblocks + 255) / 256;
  if (g > 4096) g = 4096;
  philox_words_kernel<<<(unsigned)g, 256, 0, s>>>((uint32_t)seed, (uint32_t)(seed >> 32), trial,
                                                  cand, purpose, block0, nblocks,
                                                  reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t trial, uint32_t cand, uint64_t d0, int64_t n,
                           float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  normals_kernel<<<(unsigned)g, 256, 0, s>>>((uint32_t)seed, (uint32_t)(seed >> 32), trial, cand,
                                             d0, n, out);
  return cudaGetLastError();
}

}  // namespace dg
