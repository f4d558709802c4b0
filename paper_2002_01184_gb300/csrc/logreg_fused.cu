// One launch per HMC transition for Bayesian logistic regression: the tile
// function in logreg_tile.cuh, one CTA per tile of chains.
#include "logreg_tile.cuh"

namespace hmc {

namespace {

__global__ void __launch_bounds__(lr::kLrThreads) k_logreg_fused(lr::LrArgs a) {
  lr::logreg_tile(a, static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
}

}  // namespace

// The shared-memory SIMT transition wins while a gradient's data pass is
// short (launch overhead dominates the one-launch-per-operation path); for
// long data passes the tiled products of the plain path are faster (measured
// at N = 20000, D = 128: 0.39M vs 2.2M gradient evaluations/s), so single
// posteriors use it up to 2048 data rows.  Batches use the tile at any size.
constexpr int64_t kFusedMaxRows = 2048;

bool logreg_fused_supported(const hmc_target& t) {
  return t.id == HMC_T_LOGREG && t.dim <= lr::kLrMaxDim && t.n_data <= kFusedMaxRows;
}

cudaError_t logreg_fused_setup(const hmc_target&) {
  // the attribute belongs to the kernel, shared by every context: the maximum
  return cudaFuncSetAttribute(k_logreg_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(lr::logreg_smem_bytes(lr::kLrMaxDim)));
}

unsigned logreg_fused_grid(int64_t C) {
  return static_cast<unsigned>((C + lr::kLrTC - 1) / lr::kLrTC);
}

cudaError_t launch_logreg_fused_transition(const hmc_target& t, const StepArgs& a, cudaStream_t s,
                                           KernelTimer* timer) {
  lr::LrArgs la{a, t.X, t.y, static_cast<int>(t.n_data)};
  if (timer) timer->begin(s);
  k_logreg_fused<<<logreg_fused_grid(a.C), lr::kLrThreads, lr::logreg_smem_bytes(t.dim), s>>>(la);
  if (timer) timer->end(s);
  count_launch();
  return cudaGetLastError();
}

}  // namespace hmc
