// Host-side interfaces between the translation units of libhmc.
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "hmc.h"

namespace hmc {

// Kernels launched by this library in this process (host-side count).
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// CUDA-event timing of one launch in `every` of the sampler's dominant kernel,
// on the stream it runs on.  A ring of event pairs; reading sums the pairs
// recorded since the last reset.
struct KernelTimer {
  static constexpr size_t kPairs = 2048;
  int every = 0;                 // 0: off
  uint64_t seen = 0;             // dominant launches since reset
  uint64_t recorded = 0;         // pairs recorded since reset
  cudaEvent_t ev[2 * kPairs] = {};
  bool pending = false;
  bool begin(cudaStream_t s) {
    pending = false;
    if (every <= 0) return false;
    if (seen++ % static_cast<uint64_t>(every) != 0) return false;
    const size_t k = recorded % kPairs;
    if (!ev[2 * k]) {
      if (cudaEventCreate(&ev[2 * k]) != cudaSuccess) return false;
      if (cudaEventCreate(&ev[2 * k + 1]) != cudaSuccess) return false;
    }
    pending = record(ev[2 * k], s);
    return pending;
  }
  void end(cudaStream_t s) {
    if (!pending) return;
    record(ev[2 * (recorded % kPairs) + 1], s);
    ++recorded;
    pending = false;
  }
  // Inside a stream capture a plain event record is only a dependency marker;
  // the external flag makes it a real event-record node of the graph.
  static bool record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    return cudaEventRecordWithFlags(e, s, flags) == cudaSuccess;
  }
  void destroy() {
    for (auto& e : ev)
      if (e) { cudaEventDestroy(e); e = nullptr; }
  }
};

// dx = w[c] * grad log p(x_c) per row; lp_tmp [C] receives log p.
cudaError_t launch_vjp(const hmc_target& t, int64_t C, const float* x, const float* w, float* dx,
                       float* lp_tmp, void* ws, cudaStream_t s);

// Set the error text that hmc_last_error(NULL) returns on this thread.
void set_global_error(const std::string& msg);

// SM count of the current device; 152, a GB300's, when none can be queried.
int current_sm_count();

// Bytes of scratch the batched gradient of `t` needs for C chains.
size_t grad_workspace_bytes(const hmc_target& t, int64_t C);

// log p and gradient of x [C x D] into lp [C], g [C x D] with the plain
// (one GEMM per product) kernels; `ws` holds grad_workspace_bytes bytes.
cudaError_t launch_grad(const hmc_target& t, int64_t C, const float* x, float* lp, float* g,
                        void* ws, cudaStream_t s, KernelTimer* timer = nullptr);

}  // namespace hmc

namespace hmc {

struct DAState;

// Running moments of the kept states (the streaming driver), all [C x D]:
// Welford mean / m2 and, with bsize > 0, batch means -- bsum of the current
// batch and a Welford bmean / bm2 over completed batches.  mean null: off.
struct WelfordOut {
  float* mean;
  float* m2;
  int64_t bsize;
  float* bsum;
  float* bmean;
  float* bm2;
};

// Arguments shared by the transition kernels.  x, lp, g are the current state
// and its cached log-prob / gradient (updated in place on acceptance).
struct StepArgs {
  int C, D, L;
  uint64_t seed;
  uint32_t t;             // transition index (low 32 bits key the streams)
  long long t_full;       // full transition index (decides adaptation)
  uint32_t chain_offset;
  float* x;
  float* lp;
  float* g;
  DAState* da;
  double* partials;       // one double per block of the accept kernel
  uint8_t* is_accepted;   // [C]
  float* log_accept;      // [C]
  float* sample_out;      // [C x D] or null
  uint8_t* trace_acc;     // [C] or null
  float* trace_eps;       // [1] or null
  const float* betas;     // replica exchange: row r targets p^betas[r % K]; null = 1
  int K;                  // replicas per chain (1: no tempering)
  int proposal;           // hmc_proposal_kind
  WelfordOut w;           // the pair kernel updates these at kept transitions (streaming)
};

// Scratch of the plain (one launch per operation) transition.
struct PlainBuffers {
  float* xp;   // proposal position [C x D]
  float* gp;   // gradient at the proposal
  float* p;    // momentum
  float* lpp;  // log-prob at the proposal [C]
  float* h0;   // initial Hamiltonian [C]
  float* la;   // log alpha [C] (the propose / select split)
};

// NUTS (elementwise targets): per-chain scratch slots, the largest dim, and
// the most dynamic shared memory a block may take for its span starts.
constexpr int kNutsSlots = 30;
constexpr int kNutsMaxDim = 512;
constexpr size_t kNutsSpanSmemMax = 96 * 1024;
bool nuts_supported(const hmc_target& t);
size_t nuts_scratch_floats(const hmc_target& t, int64_t C);
unsigned nuts_grid(int64_t C);   // blocks of a NUTS launch (one partial sum each)
// allow the shared-memory form its dynamic shared memory (once per process)
cudaError_t nuts_prepare();
// One transition (a.t_full): state in a.x / a.lp / a.g, sample and traces at
// a.sample_out / a.trace_eps / a.trace_acc.
cudaError_t launch_nuts_transition(const hmc_target& t, const StepArgs& a, float* scratch,
                                   int max_depth, unsigned long long* leaves, cudaStream_t s,
                                   KernelTimer* timer);
// T transitions a.t_full .. a.t_full + T - 1 in one launch, none of which
// adapts the step size (T > 1); transition keep_from + k writes kept sample k
// (samples [k][C][D], trace_eps [k], trace_acc [k][C]; each may be null).
cudaError_t launch_nuts_transitions(const hmc_target& t, const StepArgs& a, float* scratch,
                                    int max_depth, unsigned long long* leaves, int T,
                                    long long keep_from, float* samples, float* trace_eps,
                                    uint8_t* trace_acc, cudaStream_t s, KernelTimer* timer);

// Largest state dimension the fused elementwise transition keeps in registers.
constexpr int kFusedElementwiseMaxDim = 1024;
// Blocks the accept / fused kernels launch for C chains (one warp per chain).
unsigned accept_blocks(int C);

cudaError_t launch_fused_elementwise(int target_id, const StepArgs& a, cudaStream_t s,
                                     KernelTimer* timer = nullptr);
cudaError_t launch_plain_transition(const hmc_target& t, const StepArgs& a, const PlainBuffers& b,
                                    void* grad_ws, cudaStream_t s, KernelTimer* timer = nullptr);
// The plain transition in two halves: the proposal with its log alpha into
// b.la, then the Metropolis-Hastings select (same arithmetic as the whole).
cudaError_t launch_plain_propose(const hmc_target& t, const StepArgs& a, const PlainBuffers& b,
                                 void* grad_ws, cudaStream_t s);
cudaError_t launch_plain_select(const StepArgs& a, const PlainBuffers& b, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                          cudaStream_t s);
cudaError_t launch_momentum(uint64_t seed, uint32_t t, int C, int D, uint32_t chain_offset,
                            float* out, cudaStream_t s);
bool logreg_fused_supported(const hmc_target& t);
cudaError_t logreg_fused_setup(const hmc_target& t);
unsigned logreg_fused_grid(int64_t C);
cudaError_t launch_logreg_fused_transition(const hmc_target& t, const StepArgs& a, cudaStream_t s,
                                           KernelTimer* timer);
// lp[r] *= beta, g[r, :] *= beta with beta = betas[r % K]
cudaError_t launch_temper(int64_t rows, int D, float* lp, float* g, const float* betas, int K,
                          cudaStream_t s);
// replica-exchange step after transition t (pairs k = t % 2, t % 2 + 2, ...)
cudaError_t launch_remc_swap(int64_t chains, int K, int D, float* x, float* lp, float* g,
                             const float* betas, uint64_t seed, uint32_t t, uint8_t* swapped,
                             cudaStream_t s);
cudaError_t launch_welford(int64_t n, const float* x, int64_t k, float* mean, float* m2,
                           int64_t bsize, float* bsum, float* bmean, float* bm2, cudaStream_t s);
cudaError_t launch_bm_ess(int64_t C, int D, int64_t K, int64_t bsize, const float* m2, const float* bmean,
                          const float* bm2, float* ess, cudaStream_t s);
cudaError_t launch_da_init(DAState* da, float eps0, int adapt, float delta, long long num_adapt,
                           cudaStream_t s);

}  // namespace hmc

#include <cuda.h>

namespace hmc {

// Device buffers and TMA descriptors of the tensor-core Gaussian path.
struct GaussTc {
  CUtensorMap mAhi[2], mAlo[2], mBhi, mBlo;
  CUtensorMap mPhi128, mPlo128;  // P head / remainder, 32 x 128 boxes
  float* Phi = nullptr;      // tf32 head / remainder of P
  float* Plo = nullptr;
  float* Ptm = nullptr;      // P in the pair kernel's tensor-memory fill order
  float* xhi[2] = {nullptr, nullptr};   // ping-pong trajectory positions
  float* xlo[2] = {nullptr, nullptr};
  float* p = nullptr;        // momentum
  float* gL = nullptr;       // gradient at the end of the trajectory
  float* lp_part = nullptr;  // [C x ntn]
  float* h0 = nullptr;       // initial Hamiltonian
  int* err = nullptr;        // device flag: a bounded wait gave up
  // dim <= 256, the pair kernel's per-thread blocks of [pairs][2][8][dim][4]
  // floats: the cached gradients, two slots of next-transition momenta, and
  // the streaming driver's running mean, m2 and batch sum
  float* pair_g = nullptr;
  float* pair_p = nullptr;
  float* pair_w = nullptr;
  // the pair kernel's acceptance statistic words (3; see gauss_pair.cu)
  unsigned long long* pair_stat = nullptr;
  int ntn = 0;
  bool fused = false;        // one launch per transition (dim <= 256)
  bool pair = false;         // ... on CTA pairs (cta_group::2)
};

// X -> tf32 head / remainder [Npad x ld] and the transposed copies [ld x Npad];
// rows >= N and columns >= D zero; y -> ypad [Npad] (logreg_tc.cu)
cudaError_t launch_lr_prepare(int N, int Npad, int D, int ld, const float* X, const float* y, float* Xhi,
                              float* Xlo, float* XThi, float* XTlo, float* ypad, cudaStream_t s);

// Logistic regression for dims the CTA-pair kernel does not take (dim > 128;
// rows padded to ld = dim rounded up to 4 inside the workspace): each
// leapfrog gradient is two one-CTA tcgen05 products (gauss_tc.cu's tile
// pipeline): Z = Theta X^T in 64-row data tiles (two CTAs per SM) with R = y - sigmoid(Z) in
// the epilogue (R to HBM as tf32 head / remainder), then G = R X in K-split
// tiles up to 256 dims wide, summed with the prior and the leapfrog update
// by k_lr_gemm_update.
struct LogregGemm {
  CUtensorMap mThi[2], mTlo[2];  // positions [C x D], 128-row boxes (A of Z)
  CUtensorMap mXhi, mXlo;        // X [Npad x D], bnz-row boxes (B of Z)
  CUtensorMap mRhi, mRlo;        // R [C x Npad], 128-row boxes (A of G)
  CUtensorMap mXThi, mXTlo;      // X^T [D x Npad], bng-row boxes (B of G)
  float* Xhi = nullptr;
  float* Xlo = nullptr;
  float* XThi = nullptr;
  float* XTlo = nullptr;
  float* ypad = nullptr;
  float* Rhi = nullptr;
  float* Rlo = nullptr;
  float* xhi[2] = {nullptr, nullptr};
  float* xlo[2] = {nullptr, nullptr};
  float* p = nullptr;
  float* gL = nullptr;
  float* lp_part = nullptr;      // [C x ntot]: row tiles' log-likelihood, then dim tiles' prior
  float* h0 = nullptr;
  int* err = nullptr;
  int npad = 0, nrt = 0, ndt = 0, ntot = 0;
  int bnz = 64, bng = 64;        // tile widths of Z (data rows) and G = R X (dims)
  int nvalid = 0;                // data rows N
  int ld = 0;                    // padded row length of the workspace arrays
  float* part = nullptr;         // split-K products of G = R X [splits x C x ld]
  int sms = 0;                   // the device's SM count (K-split decision)
};
bool logreg_gemm_supported(const hmc_target& t);
size_t logreg_gemm_workspace_bytes(const hmc_target& t, int64_t C);
cudaError_t logreg_gemm_setup(LogregGemm* g, const hmc_target& t, int64_t C, void* ws, cudaStream_t s);
cudaError_t launch_logreg_gemm_transition(const StepArgs& a, LogregGemm& g, cudaStream_t s,
                                          KernelTimer* timer);
cudaError_t launch_logreg_gemm_products(LogregGemm& g, int C, int D, const DAState* da,
                                        const uint8_t* active, int* splits, cudaStream_t s);

bool gauss_tc_supported(const hmc_target& t);
// Tensor map of [K x C x D] float32 samples, box 128 dims x 64 chains x 1
// (false: no encoder, D % 4 != 0 or a base without 16-byte alignment).
bool make_sample_map(CUtensorMap* map, const float* base, int D, int64_t C, int64_t K);
size_t gauss_tc_workspace_bytes(const hmc_target& t, int64_t C);
cudaError_t gauss_tc_setup(GaussTc* tc, const hmc_target& t, int64_t C, void* ws, cudaStream_t s);
bool gauss_fused_supported(const hmc_target& t);
unsigned gauss_pair_grid(int64_t C);
// C rounded up to whole pairs of 64 chains
inline int64_t gauss_pair_padded_chains(int64_t C) { return (C + 63) / 64 * 64; }
// floats of the pair kernel's tensor-memory image of P (dim <= 256)
constexpr size_t kGaussPairImageFloats = 2 * 6 * 2 * 2 * 4 * 4 * 32 * 4;
cudaError_t launch_gauss_pair_image(const float* Phi, const float* Plo, int D, float* image,
                                    cudaStream_t s);
cudaError_t launch_gauss_momentum(const StepArgs& a, GaussTc& tc, cudaStream_t s);
cudaError_t gauss_pair_setup();
cudaError_t launch_gauss_pair_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                         KernelTimer* timer);
// All CTA pairs for C chains resident at once: several transitions per
// (cooperative) launch are possible.
bool gauss_pair_persistent_ok(int64_t C);
// T transitions from a.t / a.t_full in one launch; transition t_full >=
// keep_from writes output k = t_full - keep_from (samples [k][C x D],
// trace_eps [k], trace_acc [k][C]; each may be null).  T > 1 needs
// gauss_pair_persistent_ok (a cooperative launch).  With swapped
// non-null (a replica set: a.betas, a.K dividing 64) every transition is
// followed by the exchange step, its flags left in swapped.
cudaError_t launch_gauss_pair_transitions(const StepArgs& a, GaussTc& tc, int T, long long keep_from,
                                          float* samples, float* trace_eps, uint8_t* trace_acc,
                                          cudaStream_t s, KernelTimer* timer, uint8_t* swapped = nullptr);
// Test support: wait limit of the pair kernel's grid barrier and a
// generation that can never complete (0: none), for every later launch.
void set_grid_barrier_debug(unsigned long long wait_ns, int unreachable_gen);
unsigned gauss_fused_grid(int64_t C);
cudaError_t gauss_fused_setup();
cudaError_t launch_gauss_fused_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                          KernelTimer* timer);
cudaError_t launch_gauss_tc_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                       KernelTimer* timer);
// NUTS on the dense targets: the gradient products of the positions in the
// first trajectory buffer (xhi[0] / xlo[0]).  `active` marks the chains still
// building their trees; a 128-chain tile with none marked is skipped.
//   Gaussian: X P into tc.gL [C x D] (the gradient is its negative).
//   Logistic regression: R = y - sigmoid(Theta X^T) with the rows'
//   log-likelihood partials in lp_part columns 0 .. nrt - 1, then the
//   *splits K-splits of R X into g.part [splits x C x ld].
cudaError_t launch_gauss_tc_product(GaussTc& tc, int C, int D, const DAState* da, const uint8_t* active,
                                    cudaStream_t s);

}  // namespace hmc

struct hmc_ctx;

namespace hmc {
// Step arguments of context `ctx` for state x at transition t (no traces).
StepArgs ctx_step_args(hmc_ctx* ctx, float* x, uint64_t t);
// hmc_bootstrap of `ctx` enqueued on stream s instead of its own stream.
hmc_status ctx_bootstrap_on(hmc_ctx* ctx, const float* x0, cudaStream_t s);
}  // namespace hmc

namespace hmc {

// Buffers and TMA descriptors of the tensor-core logistic-regression path.
struct LogregTc {
  CUtensorMap mThi, mTlo, mXhi, mXlo, mXThi, mXTlo;
  float *Xhi = nullptr, *Xlo = nullptr, *XThi = nullptr, *XTlo = nullptr, *ypad = nullptr;
  float *thi = nullptr, *tlo = nullptr, *p = nullptr, *gL = nullptr, *lpL = nullptr, *h0 = nullptr;
  float *Gpart = nullptr, *lp_part = nullptr;
  int npad = 0, ntiles = 0, nsplit = 0, tps = 0, groups = 0, dpad = 0, n_data = 0;
  int ld = 0;     // row length of the [C x ld] / [Npad x ld] arrays: dim rounded up to 4
};

bool logreg_tc_supported(const hmc_target& t);
size_t logreg_tc_workspace_bytes(const hmc_target& t, int64_t C);
cudaError_t logreg_tc_setup(LogregTc* tc, const hmc_target& t, int64_t C, void* ws, cudaStream_t s);
cudaError_t launch_logreg_tc_transition(const StepArgs& a, LogregTc& tc, int* err, cudaStream_t s,
                                        KernelTimer* timer);
// NUTS: one gradient of the positions in tc.thi / tc.tlo into the per-range
// partials tc.Gpart [nsplit x C x D] and tc.lp_part [nsplit x C]; CTA pairs
// whose 256 chains have no flag set in `active` are skipped.
cudaError_t launch_logreg_tc_grad(LogregTc& tc, int C, int D, const uint8_t* active, int* err, cudaStream_t s);

}  // namespace hmc

namespace hmc {

// NUTS on the dense targets (nuts_dense.cu): the chains advance one leaf per
// iteration of a CUDA-graph WHILE node; see that file.
struct NutsDense {
  int mode = 0;                   // 0: Gaussian (GaussTc products), 1: logistic regression
                                  // (LogregGemm products), 2: logistic regression (LogregTc pairs)
  GaussTc* tc = nullptr;
  LogregGemm* lrg = nullptr;
  LogregTc* lrtc = nullptr;
  void* chains = nullptr;         // per-chain tree state [C]
  uint8_t* active = nullptr;      // [C] chains still building their trees
  unsigned* ctr = nullptr;        // [8] leaf-loop counters: [0-2] the graph loop's, [3] the
                                  // persistent loop's grid barrier, [4-5] its chains left
  int* err = nullptr;             // the products' flag; 2: the leaf loop ran past its bound
  float* scratch = nullptr;       // [C][kNutsSlots][ld]
  unsigned long long* leaves = nullptr;   // leapfrog steps of the chains (useful gradients)
  unsigned long long* iters = nullptr;    // leaf iterations (batched gradients) so far
  int max_depth = 10;
  cudaStream_t side = nullptr;    // stream the loop body is captured on
};
bool nuts_dense_supported(const hmc_target& t);
size_t nuts_dense_chain_bytes(int64_t C);
cudaError_t nuts_dense_prepare();
// One transition; `s` must be capturing into a graph (the leaf loop is a
// conditional node of it).  sample_out / trace_acc / trace_eps of `a` are
// this transition's output rows or null.
cudaError_t launch_nuts_dense_transition(const hmc_target& t, const StepArgs& a, NutsDense& nd, cudaStream_t s,
                                         KernelTimer* timer);

}  // namespace hmc
