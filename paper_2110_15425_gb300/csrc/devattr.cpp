// Per-device launch attributes: the multiprocessor count and the dynamic
// shared-memory limit of each kernel. Both are properties of a device, so a
// process whose contexts live on several GPUs keeps one entry per device.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "dg_internal.h"

namespace dg {

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sms[kMaxDevices] = {};
std::map<std::pair<const void*, int>, int> g_smem;   // (kernel, device) -> limit set

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  return dev;
}

}  // namespace

int num_sms() {
  const int dev = current_device();
  std::lock_guard<std::mutex> g(g_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
  }
  if (g_sms[dev] == 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = sms > 0 ? sms : 1;
  }
  return g_sms[dev];
}

cudaError_t smem_limit(const void* fn, int bytes) {
  const int dev = current_device();
  std::lock_guard<std::mutex> g(g_mu);
  auto key = std::make_pair(fn, dev);
  auto it = g_smem.find(key);
  if (it != g_smem.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  g_smem[key] = bytes;
  return cudaSuccess;
}

}  // namespace dg
