// Batched target log-prob and gradient for callers that cannot allocate
// device memory.
//
// Some callers of this library must not call cudaMalloc (or any routine that
// allocates) when they evaluate a gradient: a host process that owns the
// whole device-memory budget -- for example a sampling server that reserves
// HBM up front for the resident chain state of every admitted job and
// accounts for each byte -- or a latency-critical loop where cudaMalloc's
// implicit device synchronisation would stall work on other streams.  The
// regular entry point asks the caller for scratch; this one takes its scratch
// from a fixed array in the library's own device image instead, so the caller
// passes only inputs and outputs.
//
// The array (kNoAllocScratchBytes) is part of the module: every GPU that
// loads the library holds it until the process exits.  Host code cannot use
// the array's name as a device address, so the first call on each device
// (with that device current) resolves the address with cudaGetSymbolAddress
// and caches it; that first call should come before any stream capture.
// The cached address belongs to the device's primary context: cudaDeviceReset
// destroys that context and unloads the module, after which the cached
// address is stale (the header tells callers not to use this entry point
// again after a reset).
// Every call on a device shares the one array and it keeps the last call's
// contents; nothing in it needs to start at zero (each kernel writes every
// scratch element it later reads), but calls whose kernels overlap on the
// GPU race on it and must be serialised by the caller (one stream, or events).
#include <mutex>
#include <string>

#include "hmc_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = static_cast<size_t>(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_device_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_on_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_device_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_device_scratch[dev] = p;
  }
  *out = g_device_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" hmc_status hmc_target_log_prob_and_grad_noalloc(const hmc_target* target,
                                                           int64_t num_chains, const float* x,
                                                           float* lp, float* grad,
                                                           void* cuda_stream) {
  uint64_t need = 0;
  hmc_status st = hmc_grad_workspace_bytes(target, num_chains, &need);
  if (st != HMC_OK) return st;                    // error text already set
  if (!x || !lp || !grad) {
    hmc::set_global_error("x, lp and grad must be non-NULL");
    return HMC_E_INVALID;
  }
  if (need > kNoAllocScratchBytes) {
    hmc::set_global_error("this request needs " + std::to_string(need) +
                          " bytes of scratch; the no-allocation entry point has " +
                          std::to_string(kNoAllocScratchBytes) +
                          " (use hmc_target_log_prob_and_grad with a caller workspace)");
    return HMC_E_INVALID;
  }
  void* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) {
    hmc::set_global_error(std::string("scratch set-up: ") + cudaGetErrorString(e));
    return HMC_E_CUDA;
  }
  e = hmc::launch_grad(*target, num_chains, x, lp, grad, scratch,
                       static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    hmc::set_global_error(std::string("gradient launch: ") + cudaGetErrorString(e));
    return HMC_E_CUDA;
  }
  return HMC_OK;
}
