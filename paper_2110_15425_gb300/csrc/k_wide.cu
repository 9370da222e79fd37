// Wide multitask network (stimulus + task one-hot -> hidden -> response).
#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {

cudaError_t launch_wide(const WideParams& p, int mode, const LaunchCfg& cfg, cudaStream_t s) {
  (void)p;
  (void)mode;
  (void)cfg;
  (void)s;
  return cudaErrorNotSupported;
}

}  // namespace dg
