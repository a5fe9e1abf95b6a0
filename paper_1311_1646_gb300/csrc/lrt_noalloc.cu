// sigma_noalloc: the sigma entry point for callers that must not allocate GPU
// memory.  Such callers exist: a host program that hands the whole device to its
// own memory pool (a framework caching allocator, a serving engine) and forbids
// other cudaMalloc/cudaFree traffic; a latency-critical loop that cannot afford
// the device-wide synchronization a cudaMalloc/cudaFree may cause; code that runs
// where the CUDA runtime allocator may not be entered at all.  The regular
// sigma() allocates its intermediates on first use of a (site, nsite, nvec)
// combination; this variant keeps them in a fixed static device array instead.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/lrt.h"

namespace lrt {
// implemented in lrt_host.cpp: launch an existing sigma plan with the given workspace
int sigma_launch_existing_plan(lrt_ctx* ctx, int site, int nsite, int nvec, const double* x_dev,
                               double* y_dev, double* workspace, int64_t workspace_doubles);
int ctx_device(lrt_ctx* ctx);
void ctx_set_error(lrt_ctx* ctx, const std::string& msg);
}  // namespace lrt

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[LRT_NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch, resolved once per device.  In host code the
// array's name only stands for the symbol: the address must come from
// cudaGetSymbolAddress with that device current.
static double* g_scratch_ptr[LRT_NOALLOC_MAX_DEVICES] = {nullptr};

extern "C" int sigma_noalloc(lrt_t ctx, int site, int nsite, int nvec, const double* x_dev, double* y_dev) {
  if (!ctx) return LRT_EINVAL;
  const int dev = lrt::ctx_device(ctx);
  if (dev < 0 || dev >= LRT_NOALLOC_MAX_DEVICES) {
    lrt::ctx_set_error(ctx, "sigma_noalloc: device index beyond LRT_NOALLOC_MAX_DEVICES");
    return LRT_EINVAL;
  }
  if (cudaSetDevice(dev) != cudaSuccess) {
    lrt::ctx_set_error(ctx, "sigma_noalloc: cudaSetDevice failed");
    return LRT_ECUDA;
  }
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      lrt::ctx_set_error(ctx, std::string("sigma_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return LRT_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return lrt::sigma_launch_existing_plan(ctx, site, nsite, nvec, x_dev, y_dev, g_scratch_ptr[dev],
                                         (int64_t)LRT_NOALLOC_SCRATCH_DOUBLES);
}
