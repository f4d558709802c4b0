// C ABI of libhmc (include/hmc.h): argument checking, the context's device
// workspace, and the sample_chain driver (Section 4.2) that enqueues one
// transition per step on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "hmc_device.cuh"
#include "hmc_internal.h"

using hmc::DAState;
using hmc::PlainBuffers;
using hmc::StepArgs;

struct hmc_ctx {
  hmc_target target{};
  int64_t C = 0;
  hmc_config cfg{};
  cudaStream_t stream = nullptr;
  // kernel results (Section 4.1): cached log-prob and gradient of the state
  float* lp = nullptr;
  float* g = nullptr;
  uint8_t* is_accepted = nullptr;
  float* log_accept = nullptr;
  DAState* da = nullptr;
  double* partials = nullptr;
  PlainBuffers plain{};
  void* grad_ws = nullptr;
  size_t grad_ws_bytes = 0;
  bool bootstrapped = false;
  // device staging for hmc_sample_chain_host, grown on demand
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // hmc_sample_chain_host: kept samples leave on the copy streams, segment
  // by segment, while the next segment's transitions run
  cudaStream_t copy_stream[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t seg_ready = nullptr;
  cudaEvent_t copies_done = nullptr;
  std::vector<void*> allocations;
  uint64_t device_bytes = 0;    // bytes requested from the device allocator
  hmc::KernelTimer timer;
  bool use_tc = false;          // tensor-core Gaussian path
  hmc::GaussTc tc;
  float* nuts_scratch = nullptr;           // NUTS: trajectory ends, candidates, span starts
  // NUTS: [0] leapfrog steps so far, [1] leaf steps on the schedule's
  // critical path so far, [2] the running launch's longest chain (scratch)
  unsigned long long* nuts_leaves = nullptr;
  bool nuts_dense = false;      // NUTS on a dense target: lockstep leaves, tensor-core products
  hmc::NutsDense nd;
  int64_t dom_transitions = 1;   // transitions per launch of the dominant kernel (last chain)
  bool use_lrtc = false;        // tensor-core logistic-regression path (CTA pairs, dim <= 128)
  hmc::LogregTc lrtc;
  bool use_lrgemm = false;      // tensor-core logistic regression, one-CTA tile products (dim > 128)
  hmc::LogregGemm lrg;
  int* lr_err = nullptr;
  // replica exchange (Section 2.2): K replicas per chain, rows c*K + k
  int K = 1;
  int64_t outer_chains = 0;
  float* betas = nullptr;        // device [K]
  uint8_t* swapped = nullptr;    // device [outer_chains x (K - 1)]
  // sample_chain captured as one CUDA graph, replayed while the arguments match
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  float* g_x = nullptr;
  int64_t g_B = -1, g_K = -1;
  float* g_samples = nullptr;
  float* g_eps = nullptr;
  uint8_t* g_acc = nullptr;
  uint64_t g_launches = 0;      // kernels per replay
  uint64_t g_dominant = 0;      // dominant-kernel launches per replay
  uint64_t g_recorded = 0;      // timed event pairs inside the graph
  float* g_mean = nullptr;
  float* g_m2 = nullptr;
  int64_t g_bsize = 0;
  // streaming-expectations outputs of the call in progress (null: none)
  float* s_mean = nullptr;
  float* s_m2 = nullptr;
  // batch means of the streaming call in progress (s_bsize 0: none); the
  // three [chains x dim] buffers are allocated on first use
  int64_t s_bsize = 0;
  float* bm_sum = nullptr;
  float* bm_mean = nullptr;
  float* bm_m2 = nullptr;
  std::string err;
};

namespace {

thread_local std::string g_global_err;

// kept-sample segments of hmc_sample_chain_host: at least this many bytes
// each, at most this many segments; each segment's copy is split over this
// many streams (a single device-to-host copy measured 32-100 GB/s on the
// same workload, below what the link carries)
constexpr size_t kSegmentBytes = 256ull << 20;
constexpr int64_t kMaxSegments = 16;
constexpr int kCopyStreams = 4;
static_assert(sizeof(hmc_ctx::copy_stream) / sizeof(cudaStream_t) == kCopyStreams, "copy streams");

bool host_pinned(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

hmc_status fail(hmc_ctx* ctx, hmc_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_global_err = msg;
  return st;
}

hmc_status cuda_fail(hmc_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, HMC_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// The target's family, sizes and chain count (not its data pointers).
bool valid_target_shape(const hmc_target* t, int64_t C, std::string* why) {
  if (!t) { *why = "target is NULL"; return false; }
  if (t->dim < 1) { *why = "target dim must be >= 1"; return false; }
  if (C < 1) { *why = "num_chains must be >= 1"; return false; }
  if (C > (1ll << 30)) { *why = "num_chains must be <= 2^30"; return false; }
  if (C * static_cast<int64_t>(t->dim) > (1ll << 40)) { *why = "chains x dim too large"; return false; }
  switch (t->id) {
    case HMC_T_STD_NORMAL: return true;
    case HMC_T_FUNNEL:
      if (t->dim < 2) { *why = "funnel needs dim >= 2"; return false; }
      return true;
    case HMC_T_CORR_GAUSS: return true;
    case HMC_T_LOGREG:
      if (t->n_data < 1 || t->n_data > (1ll << 31) - 1) { *why = "LOGREG n_data out of range"; return false; }
      if (C * t->n_data > (1ll << 40)) { *why = "chains x n_data too large"; return false; }
      return true;
    default:
      *why = "unknown target id";
      return false;
  }
}

bool valid_target(const hmc_target* t, int64_t C, std::string* why) {
  if (!t) { *why = "target is NULL"; return false; }
  if (t->dim < 1) { *why = "target dim must be >= 1"; return false; }
  if (C < 1) { *why = "num_chains must be >= 1"; return false; }
  if (C > (1ll << 30)) { *why = "num_chains must be <= 2^30"; return false; }
  if (C * static_cast<int64_t>(t->dim) > (1ll << 40)) { *why = "chains x dim too large"; return false; }
  switch (t->id) {
    case HMC_T_STD_NORMAL: return true;
    case HMC_T_FUNNEL:
      if (t->dim < 2) { *why = "funnel needs dim >= 2"; return false; }
      return true;
    case HMC_T_CORR_GAUSS:
      if (!t->P) { *why = "CORR_GAUSS needs P"; return false; }
      return true;
    case HMC_T_LOGREG:
      if (!t->X || !t->y) { *why = "LOGREG needs X and y"; return false; }
      if (t->n_data < 1 || t->n_data > (1ll << 31) - 1) { *why = "LOGREG n_data out of range"; return false; }
      if (C * t->n_data > (1ll << 40)) { *why = "chains x n_data too large"; return false; }
      return true;
    default:
      *why = "unknown target id";
      return false;
  }
}

bool valid_config(const hmc_config* c, int64_t C, std::string* why) {
  if (!c) { *why = "config is NULL"; return false; }
  if (c->num_leapfrog < 1) { *why = "num_leapfrog must be >= 1"; return false; }
  if (!std::isfinite(c->step_size) || !(c->step_size > 0.f)) {
    *why = "step_size must be finite and > 0";
    return false;
  }
  if (c->adapt != 0 && c->adapt != 1) { *why = "adapt must be 0 or 1"; return false; }
  if (c->adapt && !(c->target_accept > 0.f && c->target_accept < 1.f)) {
    *why = "target_accept must be in (0, 1)";
    return false;
  }
  if (c->num_adapt_steps < 0) { *why = "num_adapt_steps must be >= 0"; return false; }
  if (c->impl != HMC_IMPL_FUSED && c->impl != HMC_IMPL_PLAIN && c->impl != HMC_IMPL_FUSED_SINGLE_CTA &&
      c->impl != HMC_IMPL_FUSED_TENSOR && c->impl != HMC_IMPL_FUSED_SIMT) {
    *why = "unknown impl";
    return false;
  }
  if (c->use_graph != 0 && c->use_graph != 1) { *why = "use_graph must be 0 or 1"; return false; }
  if (c->max_transitions_per_launch < 0) { *why = "max_transitions_per_launch must be >= 0"; return false; }
  if (c->proposal != HMC_PROPOSAL_LEAPFROG && c->proposal != HMC_PROPOSAL_RANDOM_WALK &&
      c->proposal != HMC_PROPOSAL_NUTS) {
    *why = "unknown proposal";
    return false;
  }
  if (c->proposal == HMC_PROPOSAL_NUTS && c->num_leapfrog > 10) {
    *why = "num_leapfrog (the NUTS maximum tree depth) must be <= 10";
    return false;
  }
  if (c->chain_offset < 0 || c->chain_offset + C > (1ll << 32)) {
    *why = "chain_offset + num_chains must fit in 32 bits";
    return false;
  }
  return true;
}

// Workspace comes from the stream-ordered allocator on the context's stream:
// creating and destroying contexts (a server admits and retires jobs all the
// time) then never synchronises the device, as cudaMalloc / cudaFree can.
template <typename T>
cudaError_t ctx_alloc(hmc_ctx* ctx, T** p, size_t count) {
  void* v = nullptr;
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMallocAsync(&v, bytes, ctx->stream);
  if (e == cudaSuccess) {
    ctx->allocations.push_back(v);
    ctx->device_bytes += bytes;
    *p = static_cast<T*>(v);
  }
  return e;
}

// Which paths a context takes and what hmc_create allocates for them: one
// function, so that the size query (hmc_create_device_bytes) and hmc_create
// cannot disagree.
struct CreatePlan {
  hmc_config cfg;          // the configuration as the context keeps it
  bool use_tc = false, tc_fused = false, tc_pair = false;
  bool use_lrtc = false, use_lrgemm = false;
  bool fused_logreg = false, fused_elementwise = false, plain_buffers = false;
  bool nuts_dense = false;
  size_t grad_ws = 0;
  uint64_t bytes = 0;      // sum of the allocation requests, each at least 16 bytes
};

CreatePlan plan_create(const hmc_target& t, int64_t num_chains, const hmc_config& config) {
  CreatePlan q;
  q.cfg = config;
  // the random walk and NUTS run the plain path's buffers (their proposals
  // are one elementwise op or their own kernel)
  if (q.cfg.proposal != HMC_PROPOSAL_LEAPFROG) q.cfg.impl = HMC_IMPL_PLAIN;
  const bool fused = q.cfg.impl != HMC_IMPL_PLAIN;
  const size_t C = static_cast<size_t>(num_chains), D = static_cast<size_t>(t.dim);
  auto add = [&](size_t b) { q.bytes += std::max<size_t>(b, 16); };
  const unsigned nblk = std::max({hmc::accept_blocks(static_cast<int>(num_chains)),
                                  hmc::gauss_fused_grid(num_chains), hmc::gauss_pair_grid(num_chains),
                                  hmc::logreg_fused_grid(num_chains), hmc::nuts_grid(num_chains)});
  add(4 * C);                        // log p
  add(4 * C * D);                    // gradient
  add(C);                            // is_accepted
  add(4 * C);                        // log alpha
  add(sizeof(DAState));
  add(8 * 2 * static_cast<size_t>(nblk));   // partial sums, two transitions' worth
  if (q.cfg.proposal == HMC_PROPOSAL_NUTS) {
    add(4 * hmc::nuts_scratch_floats(t, num_chains));
    add(3 * sizeof(unsigned long long));
    // dense targets: the tensor-core products' workspace, the trees' state,
    // the active flags, the loop counters and the iteration count
    q.nuts_dense = (t.id == HMC_T_CORR_GAUSS || t.id == HMC_T_LOGREG) && hmc::nuts_dense_supported(t);
    if (q.nuts_dense) {
      if (t.id == HMC_T_CORR_GAUSS) {
        q.use_tc = true;
        add(hmc::gauss_tc_workspace_bytes(t, num_chains));
      } else if (hmc::logreg_tc_supported(t)) {
        q.use_lrtc = true;       // dim <= 128, a multiple of 4: the CTA-pair kernel
        add(hmc::logreg_tc_workspace_bytes(t, num_chains));
        add(sizeof(int));
      } else {
        q.use_lrgemm = true;
        add(hmc::logreg_gemm_workspace_bytes(t, num_chains));
      }
      add(hmc::nuts_dense_chain_bytes(num_chains));
      add(C);
      add(8 * sizeof(unsigned));
      q.grad_ws = hmc::grad_workspace_bytes(t, num_chains);
      if (q.grad_ws) add(q.grad_ws);
      return q;
    }
  }
  q.use_tc = fused && hmc::gauss_tc_supported(t);
  if (q.use_tc) {
    add(hmc::gauss_tc_workspace_bytes(t, num_chains));
    q.tc_fused = hmc::gauss_fused_supported(t);
    q.tc_pair = q.tc_fused && q.cfg.impl != HMC_IMPL_FUSED_SINGLE_CTA;
  }
  // logistic regressions with long data passes or much work per gradient
  // (chains x rows x dim above 2^22): tensor-core products; small ones: the
  // shared-memory SIMT transition
  // A context whose shared-memory grid (one CTA per 8 chains) covers under
  // half of the SMs streams each gradient's data pass through few SMs, at
  // about 9e9 multiply-adds/s per CTA (8 chains x 2000 rows x 128 dims:
  // 0.46 ms per leapfrog step): from 10^4 data entries on, the tensor-core
  // products' fixed ~15 us per gradient costs less.
  const bool lr_narrow = t.id == HMC_T_LOGREG && (num_chains + 7) / 8 < hmc::current_sm_count() / 2 &&
                         t.n_data * t.dim > 10000;
  const bool lr_big = t.id == HMC_T_LOGREG &&
                      (t.n_data > 2048 || num_chains * t.n_data * t.dim > (1ll << 22) || lr_narrow);
  // (HMC_IMPL_FUSED_TENSOR and _SIMT fix the choice, for the batch's autotuner)
  const bool lr_tensor = (q.cfg.impl == HMC_IMPL_FUSED && lr_big) || q.cfg.impl == HMC_IMPL_FUSED_TENSOR;
  q.use_lrtc = lr_tensor && hmc::logreg_tc_supported(t);
  if (q.use_lrtc) {
    add(hmc::logreg_tc_workspace_bytes(t, num_chains));
    add(sizeof(int));
  }
  // long data passes the pair kernel does not take (dim > 128 or not a
  // multiple of 4): one-CTA tensor-core products
  q.use_lrgemm = lr_tensor && !q.use_lrtc && hmc::logreg_gemm_supported(t);
  if (q.use_lrgemm) add(hmc::logreg_gemm_workspace_bytes(t, num_chains));
  q.fused_logreg = fused && !q.use_lrtc && !q.use_lrgemm && hmc::logreg_fused_supported(t);
  q.fused_elementwise = fused && (t.id == HMC_T_STD_NORMAL || t.id == HMC_T_FUNNEL) &&
                        t.dim <= hmc::kFusedElementwiseMaxDim;
  q.plain_buffers = !q.fused_elementwise && !q.use_tc;
  if (q.plain_buffers) {
    add(4 * C * D);
    add(4 * C * D);
    add(4 * C * D);
    add(4 * C);
    add(4 * C);
    add(4 * C);
  }
  q.grad_ws = hmc::grad_workspace_bytes(t, num_chains);
  if (q.grad_ws) add(q.grad_ws);
  return q;
}

void drop_graph(hmc_ctx* ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
  ctx->g_B = ctx->g_K = -1;
}

void release(hmc_ctx* ctx) {
  drop_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  ctx->cap_stream = nullptr;
  for (cudaStream_t& cs : ctx->copy_stream) {
    if (cs) cudaStreamDestroy(cs);
    cs = nullptr;
  }
  if (ctx->nd.side) cudaStreamDestroy(ctx->nd.side);
  ctx->nd.side = nullptr;
  if (ctx->seg_ready) cudaEventDestroy(ctx->seg_ready);
  ctx->seg_ready = nullptr;
  if (ctx->copies_done) cudaEventDestroy(ctx->copies_done);
  ctx->copies_done = nullptr;
  for (void* p : ctx->allocations) cudaFreeAsync(p, ctx->stream);
  ctx->allocations.clear();
  if (ctx->stage) cudaFreeAsync(ctx->stage, ctx->stream);
  ctx->stage = nullptr;
}

bool fused_impl(const hmc_ctx* ctx) {
  return ctx->cfg.impl != HMC_IMPL_PLAIN;
}

bool uses_fused_logreg(const hmc_ctx* ctx) {
  return fused_impl(ctx) && !ctx->use_lrtc && !ctx->use_lrgemm && hmc::logreg_fused_supported(ctx->target);
}

bool uses_fused_elementwise(const hmc_ctx* ctx) {
  return fused_impl(ctx) &&
         (ctx->target.id == HMC_T_STD_NORMAL || ctx->target.id == HMC_T_FUNNEL) &&
         ctx->target.dim <= hmc::kFusedElementwiseMaxDim;
}

StepArgs make_args(hmc_ctx* ctx, float* x, uint64_t t) {
  StepArgs a{};
  a.C = static_cast<int>(ctx->C);
  a.D = ctx->target.dim;
  a.L = ctx->cfg.num_leapfrog;
  a.seed = ctx->cfg.seed;
  a.t = static_cast<uint32_t>(t);
  a.t_full = static_cast<long long>(t);
  a.chain_offset = static_cast<uint32_t>(ctx->cfg.chain_offset);
  a.x = x;
  a.lp = ctx->lp;
  a.g = ctx->g;
  a.da = ctx->da;
  a.partials = ctx->partials;
  a.is_accepted = ctx->is_accepted;
  a.log_accept = ctx->log_accept;
  a.betas = ctx->betas;
  a.K = ctx->K;
  a.proposal = ctx->cfg.proposal;
  return a;
}

cudaError_t enqueue_transition(hmc_ctx* ctx, const StepArgs& a) {
  if (ctx->nuts_dense)      // (the stream is capturing: see run_captured)
    return hmc::launch_nuts_dense_transition(ctx->target, a, ctx->nd, ctx->stream, &ctx->timer);
  if (ctx->cfg.proposal == HMC_PROPOSAL_NUTS)
    return hmc::launch_nuts_transition(ctx->target, a, ctx->nuts_scratch, ctx->cfg.num_leapfrog,
                                       ctx->nuts_leaves, ctx->stream, &ctx->timer);
  if (ctx->use_tc) return hmc::launch_gauss_tc_transition(a, ctx->tc, ctx->stream, &ctx->timer);
  if (ctx->use_lrtc)
    return hmc::launch_logreg_tc_transition(a, ctx->lrtc, ctx->lr_err, ctx->stream, &ctx->timer);
  if (ctx->use_lrgemm) return hmc::launch_logreg_gemm_transition(a, ctx->lrg, ctx->stream, &ctx->timer);
  if (uses_fused_logreg(ctx))
    return hmc::launch_logreg_fused_transition(ctx->target, a, ctx->stream, &ctx->timer);
  if (uses_fused_elementwise(ctx))
    return hmc::launch_fused_elementwise(ctx->target.id, a, ctx->stream, &ctx->timer);
  return hmc::launch_plain_transition(ctx->target, a, ctx->plain, ctx->grad_ws, ctx->stream,
                                      &ctx->timer);
}

// After a stream synchronisation: report a bounded device wait that gave up.
hmc_status check_device_flag(hmc_ctx* ctx) {
  if (!ctx->use_tc && !ctx->use_lrtc && !ctx->use_lrgemm) return HMC_OK;
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, ctx->use_tc ? ctx->tc.err : ctx->use_lrtc ? ctx->lr_err : ctx->lrg.err,
                                  sizeof(int),
                                  cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read device error flag");
  if (flag == 2 && ctx->nuts_dense)
    return fail(ctx, HMC_E_TIMEOUT, "the NUTS leaf loop ran past 2^max_depth iterations and was stopped");
  if (flag)
    return fail(ctx, HMC_E_TIMEOUT,
                "a tensor-core kernel's bounded wait gave up (site " + std::to_string(flag) + ")");
  return HMC_OK;
}

hmc_status bootstrap(hmc_ctx* ctx, const float* x0) {
  cudaError_t e = hmc::launch_grad(ctx->target, ctx->C, x0, ctx->lp, ctx->g, ctx->grad_ws, ctx->stream);
  if (e == cudaSuccess && ctx->K > 1)
    e = hmc::launch_temper(ctx->C, ctx->target.dim, ctx->lp, ctx->g, ctx->betas, ctx->K, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bootstrap gradient");
  e = hmc::launch_da_init(ctx->da, ctx->cfg.step_size, ctx->cfg.adapt, ctx->cfg.target_accept,
                          ctx->cfg.adapt ? ctx->cfg.num_adapt_steps : 0, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "dual-averaging init");
  ctx->bootstrapped = true;
  return HMC_OK;
}

// Work whose enqueueing needs a capturing stream (the dense NUTS leaf loop is
// a conditional graph node): run `body` directly when the context's stream
// is capturing already (the sample_chain graph, or a caller's capture);
// otherwise capture it on the private stream, then instantiate, launch on
// the context's stream and release the graph (freed when it completes).
template <typename F>
hmc_status run_captured(hmc_ctx* ctx, F&& body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(ctx->stream, &cs);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "capture query");
  if (cs == cudaStreamCaptureStatusActive) return body();
  if (!ctx->cap_stream) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap_stream;
  e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    ctx->stream = user;
    return cuda_fail(ctx, e, "begin capture");
  }
  hmc_status st = body();
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ctx->cap_stream, &g);
  ctx->stream = user;
  if (st != HMC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
  e = cudaGraphLaunch(ex, user);
  cudaGraphExecDestroy(ex);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
  return HMC_OK;
}

// Transitions t_begin .. t_end - 1 of a chain with B burn-in transitions
// (transition B + k writes kept sample k - out0 of the output buffers), after
// the bootstrap.
hmc_status enqueue_range(hmc_ctx* ctx, float* x, int64_t B, int64_t t_begin, int64_t t_end,
                         float* samples, float* trace_eps, uint8_t* trace_acc, int64_t out0 = 0) {
  if (ctx->nuts_dense) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(ctx->stream, &cs);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture query");
    if (cs != cudaStreamCaptureStatusActive)
      return run_captured(ctx, [&] {
        return enqueue_range(ctx, x, B, t_begin, t_end, samples, trace_eps, trace_acc, out0);
      });
  }
  const int64_t CD = ctx->C * ctx->target.dim;
  // dense Gaussian on CTA pairs: the chain's transitions in as few launches
  // as allowed (all of them in one cooperative launch by default)
  ctx->dom_transitions = 1;
  const int64_t T = t_end - t_begin;
  const int64_t cap = ctx->cfg.max_transitions_per_launch > 0
                          ? std::min<int64_t>(ctx->cfg.max_transitions_per_launch, 1ll << 30)
                          : (1ll << 30);
  const int64_t chunk = std::min(std::max<int64_t>(T, 1), cap);
  // (the streaming driver's moments are updated inside the launch)
  // (replica sets whose size divides a pair's 64 chains take the exchange
  // step inside the launch)
  const bool pair_remc = ctx->K > 1 && 64 % ctx->K == 0;
  if (ctx->use_tc && ctx->tc.pair && (ctx->K == 1 || pair_remc) && T > 0 &&
      (chunk == 1 || hmc::gauss_pair_persistent_ok(ctx->C))) {
    for (int64_t t0 = t_begin; t0 < t_end; t0 += chunk) {
      const int n = static_cast<int>(std::min(chunk, t_end - t0));
      StepArgs a = make_args(ctx, x, static_cast<uint64_t>(t0));
      if (ctx->s_mean)
        a.w = hmc::WelfordOut{ctx->s_mean, ctx->s_m2, ctx->s_bsize, ctx->bm_sum, ctx->bm_mean, ctx->bm_m2};
      cudaError_t e = hmc::launch_gauss_pair_transitions(a, ctx->tc, n, B + out0, samples, trace_eps, trace_acc,
                                                         ctx->stream, &ctx->timer, pair_remc ? ctx->swapped : nullptr);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "pair transition launch");
    }
    ctx->dom_transitions = chunk;
    return HMC_OK;
  }
  // NUTS: the transitions that do not adapt the step size run in as few
  // launches as allowed, so that each chain's tree sizes average out over
  // the run (those that adapt need every chain's statistic in between)
  int64_t t_multi = t_end;
  if (ctx->cfg.proposal == HMC_PROPOSAL_NUTS && !ctx->nuts_dense && ctx->K == 1 && !ctx->s_mean)
    t_multi = std::min<int64_t>(
        t_end, std::max<int64_t>(t_begin, ctx->cfg.adapt ? ctx->cfg.num_adapt_steps : 0));
  for (int64_t t = t_begin; t < t_multi; ++t) {
    StepArgs a = make_args(ctx, x, static_cast<uint64_t>(t));
    const int64_t k = t - B - out0;
    if (t - B >= 0) {
      a.sample_out = samples && ctx->K == 1 ? samples + k * CD : nullptr;
      a.trace_acc = trace_acc ? trace_acc + k * ctx->C : nullptr;
      a.trace_eps = trace_eps ? trace_eps + k : nullptr;
    }
    cudaError_t e = enqueue_transition(ctx, a);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "transition launch");
    if (ctx->K > 1) {
      e = hmc::launch_remc_swap(ctx->outer_chains, ctx->K, ctx->target.dim, x, ctx->lp, ctx->g,
                                ctx->betas, ctx->cfg.seed, static_cast<uint32_t>(t), ctx->swapped,
                                ctx->stream);
      if (e == cudaSuccess && k >= 0 && samples)
        e = cudaMemcpyAsync(samples + k * CD, x, CD * sizeof(float), cudaMemcpyDeviceToDevice,
                            ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "exchange step");
    }
    if (k >= 0 && ctx->s_mean) {
      e = hmc::launch_welford(CD, x, k, ctx->s_mean, ctx->s_m2, ctx->s_bsize, ctx->bm_sum, ctx->bm_mean,
                              ctx->bm_m2, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "moment update launch");
    }
  }
  for (int64_t t0 = t_multi; t0 < t_end; t0 += chunk) {
    const int n = static_cast<int>(std::min(chunk, t_end - t0));
    StepArgs a = make_args(ctx, x, static_cast<uint64_t>(t0));
    cudaError_t e = hmc::launch_nuts_transitions(ctx->target, a, ctx->nuts_scratch, ctx->cfg.num_leapfrog,
                                                 ctx->nuts_leaves, n, B + out0, samples, trace_eps, trace_acc,
                                                 ctx->stream, &ctx->timer);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "NUTS transition launch");
  }
  return HMC_OK;
}


hmc_status enqueue_chain(hmc_ctx* ctx, float* x, int64_t B, int64_t K, float* samples, float* trace_eps,
                         uint8_t* trace_acc) {
  hmc_status st = bootstrap(ctx, x);
  if (st != HMC_OK) return st;
  return enqueue_range(ctx, x, B, 0, B + K, samples, trace_eps, trace_acc);
}

// sample_chain as a CUDA graph: the first call with a given set of buffers
// and step counts captures bootstrap + every transition on a private stream;
// later calls replay the instantiated graph on the context's stream.
hmc_status run_chain(hmc_ctx* ctx, float* x, int64_t B, int64_t K, float* samples, float* trace_eps,
                     uint8_t* trace_acc) {
  if (!ctx->cfg.use_graph) return enqueue_chain(ctx, x, B, K, samples, trace_eps, trace_acc);
  const bool hit = ctx->graph && ctx->g_x == x && ctx->g_B == B && ctx->g_K == K &&
                   ctx->g_samples == samples && ctx->g_eps == trace_eps && ctx->g_acc == trace_acc &&
                   ctx->g_mean == ctx->s_mean && ctx->g_m2 == ctx->s_m2 && ctx->g_bsize == ctx->s_bsize;
  if (!hit) {
    drop_graph(ctx);
    cudaError_t e = cudaSuccess;
    if (!ctx->cap_stream) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->cap_stream;
    const uint64_t l0 = hmc::g_launches.load(), d0 = ctx->timer.seen;
    e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      ctx->stream = user;
      return cuda_fail(ctx, e, "begin capture");
    }
    hmc_status st = enqueue_chain(ctx, x, B, K, samples, trace_eps, trace_acc);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->stream = user;
    if (st != HMC_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ctx->graph = nullptr;
      return cuda_fail(ctx, e, "graph instantiate");
    }
    ctx->g_launches = hmc::g_launches.load() - l0;
    ctx->g_dominant = ctx->timer.seen - d0;
    ctx->g_recorded = ctx->timer.recorded;
    hmc::g_launches.fetch_sub(ctx->g_launches);   // counted per replay below
    ctx->timer.seen = d0;
    ctx->g_x = x;
    ctx->g_B = B;
    ctx->g_K = K;
    ctx->g_samples = samples;
    ctx->g_eps = trace_eps;
    ctx->g_acc = trace_acc;
    ctx->g_mean = ctx->s_mean;
    ctx->g_m2 = ctx->s_m2;
    ctx->g_bsize = ctx->s_bsize;
  }
  cudaError_t e = cudaGraphLaunch(ctx->graph, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
  hmc::count_launch(ctx->g_launches);
  ctx->timer.seen += ctx->g_dominant;
  // every replay re-records the event pairs captured in the graph
  ctx->timer.recorded = std::max(ctx->timer.recorded, ctx->g_recorded);
  ctx->bootstrapped = true;
  return HMC_OK;
}

}  // namespace

namespace hmc {
void set_global_error(const std::string& msg) { g_global_err = msg; }

StepArgs ctx_step_args(hmc_ctx* ctx, float* x, uint64_t t) { return make_args(ctx, x, t); }

hmc_status ctx_bootstrap_on(hmc_ctx* ctx, const float* x0, cudaStream_t s) {
  cudaStream_t own = ctx->stream;
  ctx->stream = s;
  hmc_status st = bootstrap(ctx, x0);
  ctx->stream = own;
  return st;
}
}  // namespace hmc

extern "C" {

hmc_status hmc_create(const hmc_target* target, int64_t num_chains, const hmc_config* config,
                      void* cuda_stream, hmc_ctx** out) {
  std::string why;
  if (!out) return fail(nullptr, HMC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!valid_target(target, num_chains, &why)) return fail(nullptr, HMC_E_INVALID, why);
  if (!valid_config(config, num_chains, &why)) return fail(nullptr, HMC_E_INVALID, why);
  if (config->proposal == HMC_PROPOSAL_NUTS && !hmc::nuts_supported(*target) &&
      !hmc::nuts_dense_supported(*target))
    return fail(nullptr, HMC_E_UNSUPPORTED,
                "NUTS runs targets with dim <= 512 (CORR_GAUSS: dim a multiple of 4)");
  hmc_ctx* ctx = new (std::nothrow) hmc_ctx();
  if (!ctx) return fail(nullptr, HMC_E_OOM, "host allocation failed");
  const CreatePlan plan = plan_create(*target, num_chains, *config);
  ctx->target = *target;
  ctx->C = num_chains;
  ctx->cfg = plan.cfg;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t C = static_cast<size_t>(num_chains), D = static_cast<size_t>(target->dim);
  cudaError_t e = cudaSuccess;
  // one partial sum per block of whichever transition kernel runs
  const unsigned nblk = std::max({hmc::accept_blocks(static_cast<int>(num_chains)),
                                  hmc::gauss_fused_grid(num_chains),
                                  hmc::gauss_pair_grid(num_chains),
                                  hmc::logreg_fused_grid(num_chains),
                                  hmc::nuts_grid(num_chains)});
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->lp, C);
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->g, C * D);
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->is_accepted, C);
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->log_accept, C);
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->da, 1);
  // (two transitions' worth: the multi-transition pair launch alternates)
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->partials, 2 * static_cast<size_t>(nblk));
  if (e == cudaSuccess && ctx->cfg.proposal == HMC_PROPOSAL_NUTS) {
    e = hmc::nuts_prepare();
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->nuts_scratch, hmc::nuts_scratch_floats(*target, num_chains));
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->nuts_leaves, 3);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->nuts_leaves, 0, 3 * sizeof(unsigned long long), ctx->stream);
  }
  ctx->use_tc = plan.use_tc;
  if (e == cudaSuccess && ctx->use_tc) {
    char* w = nullptr;
    e = ctx_alloc(ctx, &w, hmc::gauss_tc_workspace_bytes(*target, num_chains));
    if (e == cudaSuccess) e = hmc::gauss_tc_setup(&ctx->tc, *target, num_chains, w, ctx->stream);
    ctx->tc.fused = plan.tc_fused;
    ctx->tc.pair = plan.tc_pair;
  }
  ctx->use_lrtc = plan.use_lrtc;
  if (e == cudaSuccess && ctx->use_lrtc) {
    char* w = nullptr;
    e = ctx_alloc(ctx, &w, hmc::logreg_tc_workspace_bytes(*target, num_chains));
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->lr_err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->lr_err, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = hmc::logreg_tc_setup(&ctx->lrtc, *target, num_chains, w, ctx->stream);
  }
  ctx->use_lrgemm = plan.use_lrgemm;
  if (e == cudaSuccess && ctx->use_lrgemm) {
    char* w = nullptr;
    e = ctx_alloc(ctx, &w, hmc::logreg_gemm_workspace_bytes(*target, num_chains));
    if (e == cudaSuccess) e = hmc::logreg_gemm_setup(&ctx->lrg, *target, num_chains, w, ctx->stream);
  }
  ctx->nuts_dense = plan.nuts_dense;
  if (e == cudaSuccess && ctx->nuts_dense) {
    hmc::NutsDense& nd = ctx->nd;
    nd.mode = target->id == HMC_T_CORR_GAUSS ? 0 : ctx->use_lrtc ? 2 : 1;
    nd.tc = &ctx->tc;
    nd.lrg = &ctx->lrg;
    nd.lrtc = &ctx->lrtc;
    nd.err = nd.mode == 0 ? ctx->tc.err : nd.mode == 2 ? ctx->lr_err : ctx->lrg.err;
    nd.scratch = ctx->nuts_scratch;
    nd.leaves = ctx->nuts_leaves;
    nd.max_depth = ctx->cfg.num_leapfrog;
    char* ch = nullptr;
    e = ctx_alloc(ctx, &ch, hmc::nuts_dense_chain_bytes(num_chains));
    nd.chains = ch;
    if (e == cudaSuccess) e = ctx_alloc(ctx, &nd.active, C);
    if (e == cudaSuccess) e = ctx_alloc(ctx, &nd.ctr, 8);
    nd.iters = ctx->nuts_leaves + 1;
    if (e == cudaSuccess) e = cudaMemsetAsync(nd.ctr, 0, 8 * sizeof(unsigned), ctx->stream);
    if (e == cudaSuccess) e = hmc::nuts_dense_prepare();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&nd.side, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess && plan.fused_logreg) e = hmc::logreg_fused_setup(*target);
  if (e == cudaSuccess && plan.plain_buffers) {
    e = ctx_alloc(ctx, &ctx->plain.xp, C * D);
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->plain.gp, C * D);
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->plain.p, C * D);
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->plain.lpp, C);
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->plain.h0, C);
    if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->plain.la, C);
  }
  ctx->grad_ws_bytes = plan.grad_ws;
  if (e == cudaSuccess && ctx->grad_ws_bytes) {
    char* w = nullptr;
    e = ctx_alloc(ctx, &w, ctx->grad_ws_bytes);
    ctx->grad_ws = w;
  }
  if (e == cudaSuccess) {
    // zero the arrival counter so the first transition's grid reduction works
    // even before hmc_bootstrap re-initialises the state
    e = cudaMemsetAsync(ctx->da, 0, sizeof(DAState), ctx->stream);
  }
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    cudaGetLastError();
    release(ctx);
    delete ctx;
    return fail(nullptr, oom ? HMC_E_OOM : HMC_E_CUDA,
                std::string("workspace allocation: ") + cudaGetErrorString(e));
  }
  *out = ctx;
  return HMC_OK;
}

hmc_status hmc_create_device_bytes(const hmc_target* target, int64_t num_chains, const hmc_config* config,
                                   uint64_t* bytes) {
  std::string why;
  if (!bytes) return fail(nullptr, HMC_E_INVALID, "bytes is NULL");
  if (!valid_target_shape(target, num_chains, &why)) return fail(nullptr, HMC_E_INVALID, why);
  if (!valid_config(config, num_chains, &why)) return fail(nullptr, HMC_E_INVALID, why);
  *bytes = plan_create(*target, num_chains, *config).bytes;
  return HMC_OK;
}

hmc_status hmc_context_device_bytes(const hmc_ctx* ctx, uint64_t* bytes) {
  if (!ctx || !bytes) return fail(nullptr, HMC_E_INVALID, "NULL argument");
  *bytes = ctx->device_bytes + ctx->stage_bytes;
  return HMC_OK;
}

hmc_status hmc_bootstrap(hmc_ctx* ctx, const float* x0) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x0) return fail(ctx, HMC_E_INVALID, "x0 is NULL");
  return bootstrap(ctx, x0);
}

hmc_status hmc_step(hmc_ctx* ctx, float* x_inout, uint64_t t, hmc_kernel_results* out) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x_inout) return fail(ctx, HMC_E_INVALID, "x_inout is NULL");
  if (!ctx->bootstrapped) return fail(ctx, HMC_E_INVALID, "hmc_bootstrap must precede hmc_step");
  if (t > std::numeric_limits<uint32_t>::max())
    return fail(ctx, HMC_E_INVALID, "transition index must fit in 32 bits");
  StepArgs a = make_args(ctx, x_inout, t);
  cudaError_t e = cudaSuccess;
  if (ctx->nuts_dense) {
    hmc_status st = run_captured(ctx, [&] {
      const cudaError_t le = enqueue_transition(ctx, make_args(ctx, x_inout, t));
      return le == cudaSuccess ? HMC_OK : cuda_fail(ctx, le, "transition launch");
    });
    if (st != HMC_OK) return st;
  } else {
    e = enqueue_transition(ctx, a);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "transition launch");
  if (ctx->K > 1) {
    e = hmc::launch_remc_swap(ctx->outer_chains, ctx->K, ctx->target.dim, x_inout, ctx->lp, ctx->g,
                              ctx->betas, ctx->cfg.seed, static_cast<uint32_t>(t), ctx->swapped,
                              ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "exchange step");
  }
  if (out) {
    out->target_log_prob = ctx->lp;
    out->grad = ctx->g;
    out->is_accepted = ctx->is_accepted;
    out->log_accept_ratio = ctx->log_accept;
    out->step_size = &ctx->da->eps;
  }
  return HMC_OK;
}

namespace {
hmc_status split_ready(hmc_ctx* ctx, const void* x, uint64_t t) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x) return fail(ctx, HMC_E_INVALID, "state pointer is NULL");
  if (ctx->cfg.impl != HMC_IMPL_PLAIN || ctx->K != 1 || !ctx->plain.la ||
      ctx->cfg.proposal == HMC_PROPOSAL_NUTS)
    return fail(ctx, HMC_E_UNSUPPORTED,
                "the propose / select split needs impl = HMC_IMPL_PLAIN (or the random walk) and no replicas");
  if (!ctx->bootstrapped) return fail(ctx, HMC_E_INVALID, "hmc_bootstrap must come first");
  if (t > std::numeric_limits<uint32_t>::max())
    return fail(ctx, HMC_E_INVALID, "transition index must fit in 32 bits");
  return HMC_OK;
}
}  // namespace

hmc_status hmc_nuts_leapfrog_count(hmc_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return fail(ctx, HMC_E_INVALID, "NULL argument");
  if (ctx->cfg.proposal != HMC_PROPOSAL_NUTS || !ctx->nuts_leaves)
    return fail(ctx, HMC_E_INVALID, "the context does not run NUTS");
  unsigned long long v = 0;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, ctx->nuts_leaves, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read leapfrog count");
  *out = static_cast<uint64_t>(v);
  return HMC_OK;
}

hmc_status hmc_nuts_leaf_iterations(hmc_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return fail(ctx, HMC_E_INVALID, "NULL argument");
  if (ctx->cfg.proposal != HMC_PROPOSAL_NUTS || !ctx->nuts_leaves)
    return fail(ctx, HMC_E_INVALID, "the context does not run NUTS");
  unsigned long long v = 0;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, ctx->nuts_leaves + 1, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read leaf iterations");
  *out = static_cast<uint64_t>(v);
  return HMC_OK;
}

hmc_status hmc_propose(hmc_ctx* ctx, const float* x, uint64_t t, hmc_proposal* out) {
  hmc_status st = split_ready(ctx, x, t);
  if (st != HMC_OK) return st;
  StepArgs a = make_args(ctx, const_cast<float*>(x), t);   // read only in the proposal kernels
  cudaError_t e = hmc::launch_plain_propose(ctx->target, a, ctx->plain, ctx->grad_ws, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "proposal launch");
  if (out) {
    out->x = ctx->plain.xp;
    out->target_log_prob = ctx->plain.lpp;
    out->grad = ctx->plain.gp;
    out->log_accept_ratio = ctx->plain.la;
  }
  return HMC_OK;
}

hmc_status hmc_mh_select(hmc_ctx* ctx, float* x_inout, uint64_t t, hmc_kernel_results* out) {
  hmc_status st = split_ready(ctx, x_inout, t);
  if (st != HMC_OK) return st;
  StepArgs a = make_args(ctx, x_inout, t);
  cudaError_t e = hmc::launch_plain_select(a, ctx->plain, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "select launch");
  if (out) {
    out->target_log_prob = ctx->lp;
    out->grad = ctx->g;
    out->is_accepted = ctx->is_accepted;
    out->log_accept_ratio = ctx->log_accept;
    out->step_size = &ctx->da->eps;
  }
  return HMC_OK;
}

hmc_status hmc_sample_chain(hmc_ctx* ctx, float* x_inout, int64_t num_burnin, int64_t num_results,
                            float* samples_out, float* trace_step_size, uint8_t* trace_accept) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x_inout) return fail(ctx, HMC_E_INVALID, "x_inout is NULL");
  if (num_burnin < 0 || num_results < 0) return fail(ctx, HMC_E_INVALID, "negative step count");
  if (num_burnin + num_results > static_cast<int64_t>(std::numeric_limits<uint32_t>::max()))
    return fail(ctx, HMC_E_INVALID, "too many transitions (transition index is 32-bit)");
  return run_chain(ctx, x_inout, num_burnin, num_results, samples_out, trace_step_size, trace_accept);
}

hmc_status hmc_sample_chain_streaming(hmc_ctx* ctx, float* x_inout, int64_t num_burnin,
                                      int64_t num_results, float* mean_out, float* m2_out,
                                      float* trace_step_size, uint8_t* trace_accept) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x_inout || !mean_out || !m2_out)
    return fail(ctx, HMC_E_INVALID, "x_inout, mean_out and m2_out must be non-NULL");
  if (num_burnin < 0 || num_results < 0) return fail(ctx, HMC_E_INVALID, "negative step count");
  if (num_burnin + num_results > static_cast<int64_t>(std::numeric_limits<uint32_t>::max()))
    return fail(ctx, HMC_E_INVALID, "too many transitions (transition index is 32-bit)");
  ctx->s_mean = mean_out;
  ctx->s_m2 = m2_out;
  hmc_status st = run_chain(ctx, x_inout, num_burnin, num_results, nullptr, trace_step_size,
                            trace_accept);
  ctx->s_mean = nullptr;
  ctx->s_m2 = nullptr;
  return st;
}

hmc_status hmc_sample_chain_streaming_ess(hmc_ctx* ctx, float* x_inout, int64_t num_burnin,
                                          int64_t num_results, int64_t batch_size, float* mean_out,
                                          float* m2_out, float* ess_out, float* trace_step_size,
                                          uint8_t* trace_accept) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x_inout || !mean_out || !m2_out || !ess_out)
    return fail(ctx, HMC_E_INVALID, "x_inout, mean_out, m2_out and ess_out must be non-NULL");
  if (num_burnin < 0 || num_results < 0) return fail(ctx, HMC_E_INVALID, "negative step count");
  if (num_burnin + num_results > static_cast<int64_t>(std::numeric_limits<uint32_t>::max()))
    return fail(ctx, HMC_E_INVALID, "too many transitions (transition index is 32-bit)");
  if (batch_size < 1 || num_results / batch_size < 1 || ctx->C * (num_results / batch_size) < 2)
    return fail(ctx, HMC_E_INVALID,
                "need batch_size >= 1, one complete batch per chain and at least two batches in all");
  if (ctx->K > 1)
    return fail(ctx, HMC_E_UNSUPPORTED, "batch-means ESS pools the chains of one target, not a replica set");
  const size_t CD = static_cast<size_t>(ctx->C) * ctx->target.dim;
  cudaError_t e = cudaSuccess;
  if (!ctx->bm_sum) e = ctx_alloc(ctx, &ctx->bm_sum, CD);
  if (e == cudaSuccess && !ctx->bm_mean) e = ctx_alloc(ctx, &ctx->bm_mean, CD);
  if (e == cudaSuccess && !ctx->bm_m2) e = ctx_alloc(ctx, &ctx->bm_m2, CD);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? HMC_E_OOM : HMC_E_CUDA,
                std::string("batch-means workspace: ") + cudaGetErrorString(e));
  }
  ctx->s_mean = mean_out;
  ctx->s_m2 = m2_out;
  ctx->s_bsize = batch_size;
  hmc_status st = run_chain(ctx, x_inout, num_burnin, num_results, nullptr, trace_step_size,
                            trace_accept);
  ctx->s_mean = nullptr;
  ctx->s_m2 = nullptr;
  ctx->s_bsize = 0;
  if (st != HMC_OK) return st;
  e = hmc::launch_bm_ess(ctx->C, ctx->target.dim, num_results, batch_size, m2_out, ctx->bm_mean,
                         ctx->bm_m2, ess_out, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch-means ESS launch");
  return HMC_OK;
}

hmc_status hmc_sample_chain_host(hmc_ctx* ctx, float* x_inout, int64_t num_burnin,
                                 int64_t num_results, float* samples_out, float* trace_step_size,
                                 uint8_t* trace_accept) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x_inout) return fail(ctx, HMC_E_INVALID, "x_inout is NULL");
  if (num_burnin < 0 || num_results < 0) return fail(ctx, HMC_E_INVALID, "negative step count");
  if (num_burnin + num_results > static_cast<int64_t>(std::numeric_limits<uint32_t>::max()))
    return fail(ctx, HMC_E_INVALID, "too many transitions (transition index is 32-bit)");
  const size_t CD = static_cast<size_t>(ctx->C) * ctx->target.dim;
  const size_t K = static_cast<size_t>(num_results);
  auto a256 = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const size_t off_s = a256(CD * sizeof(float));
  const size_t off_e = off_s + (samples_out ? a256(K * CD * sizeof(float)) : 0);
  const size_t off_a = off_e + (trace_step_size ? a256(K * sizeof(float)) : 0);
  const size_t total = off_a + (trace_accept ? a256(K * ctx->C) : 0);
  if (total > ctx->stage_bytes) {
    if (ctx->stage) cudaFreeAsync(ctx->stage, ctx->stream);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    cudaError_t e = cudaMallocAsync(&ctx->stage, total, ctx->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, e == cudaErrorMemoryAllocation ? HMC_E_OOM : HMC_E_CUDA,
                  std::string("staging allocation: ") + cudaGetErrorString(e));
    }
    ctx->stage_bytes = total;
  }
  char* base = static_cast<char*>(ctx->stage);
  float* dx = reinterpret_cast<float*>(base);
  float* ds = samples_out ? reinterpret_cast<float*>(base + off_s) : nullptr;
  float* de = trace_step_size ? reinterpret_cast<float*>(base + off_e) : nullptr;
  uint8_t* dacc = trace_accept ? reinterpret_cast<uint8_t*>(base + off_a) : nullptr;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(dx, x_inout, CD * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "state upload");
  // Large sample sets bound for pinned host memory leave the device in
  // segments of kept transitions, each copied on a second stream while the
  // next segment runs; otherwise the whole chain (one CUDA graph) runs first.
  const size_t sample_bytes = K * CD * sizeof(float);
  int64_t nseg = 1;
  // (not for NUTS: its fixed-step-size run is one launch whose length is its
  // slowest chain's, and each segment would pay that chain's tail again)
  if (ds && K > 1 && ctx->cfg.proposal != HMC_PROPOSAL_NUTS &&
      sample_bytes >= 2 * kSegmentBytes && host_pinned(samples_out))
    nseg = std::min<int64_t>({kMaxSegments, static_cast<int64_t>(K),
                              static_cast<int64_t>(sample_bytes / kSegmentBytes)});
  if (nseg == 1) {
    hmc_status st = run_chain(ctx, dx, num_burnin, num_results, ds, de, dacc);
    if (st != HMC_OK) return st;
  } else {
    for (int c = 0; c < kCopyStreams && e == cudaSuccess; ++c)
      if (!ctx->copy_stream[c]) e = cudaStreamCreateWithFlags(&ctx->copy_stream[c], cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->seg_ready) e = cudaEventCreateWithFlags(&ctx->seg_ready, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->copies_done)
      e = cudaEventCreateWithFlags(&ctx->copies_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
    hmc_status st = bootstrap(ctx, dx);
    if (st == HMC_OK) st = enqueue_range(ctx, dx, num_burnin, 0, num_burnin, ds, de, dacc);
    for (int64_t i = 0; i < nseg && st == HMC_OK; ++i) {
      const int64_t k0 = static_cast<int64_t>(K) * i / nseg, k1 = static_cast<int64_t>(K) * (i + 1) / nseg;
      st = enqueue_range(ctx, dx, num_burnin, num_burnin + k0, num_burnin + k1, ds, de, dacc);
      if (st != HMC_OK) break;
      e = cudaEventRecord(ctx->seg_ready, s);
      // the segment's bytes in kCopyStreams contiguous pieces, one per stream
      const size_t seg0 = static_cast<size_t>(k0) * CD, seg_n = static_cast<size_t>(k1 - k0) * CD;
      for (int c = 0; c < kCopyStreams && e == cudaSuccess; ++c) {
        const size_t a0 = seg0 + seg_n * c / kCopyStreams, a1 = seg0 + seg_n * (c + 1) / kCopyStreams;
        e = cudaStreamWaitEvent(ctx->copy_stream[c], ctx->seg_ready, 0);
        if (e == cudaSuccess && a1 > a0)
          e = cudaMemcpyAsync(samples_out + a0, ds + a0, (a1 - a0) * sizeof(float), cudaMemcpyDeviceToHost,
                              ctx->copy_stream[c]);
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "sample download");
    }
    if (st != HMC_OK) return st;
    for (int c = 0; c < kCopyStreams && e == cudaSuccess; ++c) {
      e = cudaEventRecord(ctx->copies_done, ctx->copy_stream[c]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->copies_done, 0);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sample download");
  }
  e = cudaMemcpyAsync(x_inout, dx, CD * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ds && nseg == 1)
    e = cudaMemcpyAsync(samples_out, ds, K * CD * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && de)
    e = cudaMemcpyAsync(trace_step_size, de, K * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && dacc)
    e = cudaMemcpyAsync(trace_accept, dacc, K * ctx->C, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "result download");
  return check_device_flag(ctx);
}

hmc_status hmc_sample_chain_range(hmc_ctx* ctx, float* x_inout, int64_t num_burnin, int64_t t_begin,
                                  int64_t t_end, float* samples_out, float* trace_step_size,
                                  uint8_t* trace_accept) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!x_inout) return fail(ctx, HMC_E_INVALID, "x_inout is NULL");
  if (num_burnin < 0 || t_begin < 0 || t_end < t_begin)
    return fail(ctx, HMC_E_INVALID, "need num_burnin >= 0 and 0 <= t_begin <= t_end");
  if (t_end > static_cast<int64_t>(std::numeric_limits<uint32_t>::max()))
    return fail(ctx, HMC_E_INVALID, "too many transitions (transition index is 32-bit)");
  if (t_begin > 0 && !ctx->bootstrapped)
    return fail(ctx, HMC_E_INVALID, "a range that does not start at 0 needs the previous state (hmc_restore_state)");
  if (t_begin == 0) {
    hmc_status st = bootstrap(ctx, x_inout);
    if (st != HMC_OK) return st;
  }
  return enqueue_range(ctx, x_inout, num_burnin, t_begin, t_end, samples_out, trace_step_size, trace_accept,
                       std::max<int64_t>(0, t_begin - num_burnin));
}

namespace {
// Layout of a saved context state: a header, the dual-averaging state, the
// cached log p [rows] and gradient [rows x dim] (rows = chains x replicas).
struct SavedHeader {
  uint64_t magic;
  int64_t rows;
  int32_t dim, target, replicas, da_bytes;
};
constexpr uint64_t kStateMagic = 0x31544154534d4348ull;   // "HCMSTAT1"
size_t state_bytes(const hmc_ctx* ctx) {
  return sizeof(SavedHeader) + sizeof(DAState) + sizeof(float) * static_cast<size_t>(ctx->C) +
         sizeof(float) * static_cast<size_t>(ctx->C) * ctx->target.dim;
}
}  // namespace

hmc_status hmc_state_bytes(const hmc_ctx* ctx, uint64_t* bytes) {
  if (!ctx || !bytes) return fail(nullptr, HMC_E_INVALID, "NULL argument");
  *bytes = state_bytes(ctx);
  return HMC_OK;
}

hmc_status hmc_save_state(hmc_ctx* ctx, void* out, uint64_t bytes) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!out || bytes < state_bytes(ctx)) return fail(ctx, HMC_E_INVALID, "out is NULL or smaller than hmc_state_bytes");
  if (!ctx->bootstrapped) return fail(ctx, HMC_E_INVALID, "nothing to save before hmc_bootstrap");
  char* base = static_cast<char*>(out);
  SavedHeader h{kStateMagic, ctx->C, ctx->target.dim, ctx->target.id, ctx->K, static_cast<int32_t>(sizeof(DAState))};
  std::memcpy(base, &h, sizeof(h));
  char* p = base + sizeof(h);
  cudaError_t e = cudaMemcpyAsync(p, ctx->da, sizeof(DAState), cudaMemcpyDeviceToHost, ctx->stream);
  p += sizeof(DAState);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, ctx->lp, sizeof(float) * ctx->C, cudaMemcpyDeviceToHost, ctx->stream);
  p += sizeof(float) * ctx->C;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p, ctx->g, sizeof(float) * ctx->C * ctx->target.dim, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "save state");
  return check_device_flag(ctx);
}

hmc_status hmc_restore_state(hmc_ctx* ctx, const void* in, uint64_t bytes) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!in || bytes < state_bytes(ctx)) return fail(ctx, HMC_E_INVALID, "in is NULL or smaller than hmc_state_bytes");
  const char* base = static_cast<const char*>(in);
  SavedHeader h;
  std::memcpy(&h, base, sizeof(h));
  if (h.magic != kStateMagic || h.rows != ctx->C || h.dim != ctx->target.dim || h.target != ctx->target.id ||
      h.replicas != ctx->K || h.da_bytes != static_cast<int32_t>(sizeof(DAState)))
    return fail(ctx, HMC_E_INVALID, "the saved state belongs to another target, chain count or build");
  const char* p = base + sizeof(h);
  // the transfers are synchronous: the caller's buffer may be released on return
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->da, p, sizeof(DAState), cudaMemcpyHostToDevice);
  p += sizeof(DAState);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->lp, p, sizeof(float) * ctx->C, cudaMemcpyHostToDevice);
  p += sizeof(float) * ctx->C;
  if (e == cudaSuccess) e = cudaMemcpy(ctx->g, p, sizeof(float) * ctx->C * ctx->target.dim, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "restore state");
  ctx->bootstrapped = true;
  return HMC_OK;
}

void hmc_debug_set_grid_barrier(uint64_t wait_limit_ns, int32_t unreachable_generation) {
  hmc::set_grid_barrier_debug(static_cast<unsigned long long>(wait_limit_ns), unreachable_generation);
}

hmc_status hmc_read_adaptation(hmc_ctx* ctx, double out[5]) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (!out) return fail(ctx, HMC_E_INVALID, "out is NULL");
  DAState h{};
  cudaError_t e = cudaMemcpyAsync(&h, ctx->da, sizeof(DAState), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "read adaptation state");
  hmc_status st = check_device_flag(ctx);
  if (st != HMC_OK) return st;
  out[0] = static_cast<double>(h.eps);
  out[1] = h.log_eps_bar;
  out[2] = h.h_bar;
  out[3] = static_cast<double>(h.m);
  out[4] = h.last_stat;
  return HMC_OK;
}

hmc_status hmc_remc_create(const hmc_target* target, int64_t num_chains, int32_t num_replicas,
                           const float* betas, const hmc_config* config, void* cuda_stream,
                           hmc_ctx** out) {
  if (!out) return fail(nullptr, HMC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (num_replicas < 2) return fail(nullptr, HMC_E_INVALID, "num_replicas must be >= 2");
  if (!betas) return fail(nullptr, HMC_E_INVALID, "betas is NULL");
  for (int k = 0; k < num_replicas; ++k)
    if (!std::isfinite(betas[k]) || !(betas[k] > 0.f) || betas[k] > 1.f)
      return fail(nullptr, HMC_E_INVALID, "betas must lie in (0, 1]");
  if (!config) return fail(nullptr, HMC_E_INVALID, "config is NULL");
  if (config->adapt) return fail(nullptr, HMC_E_UNSUPPORTED, "replica exchange uses a fixed step size");
  if (config->proposal == HMC_PROPOSAL_NUTS)
    return fail(nullptr, HMC_E_UNSUPPORTED, "replica exchange runs the leapfrog or random-walk proposal");
  if (config->chain_offset != 0) return fail(nullptr, HMC_E_INVALID, "chain_offset must be 0");
  if (num_chains < 1 || num_chains > (1ll << 30) / num_replicas)
    return fail(nullptr, HMC_E_INVALID, "num_chains out of range");
  hmc_config c = *config;
  // Of the dense targets' tensor-core kernels only the CTA-pair Gaussian
  // kernel tempers (one launch per transition, the exchange step between
  // launches); the others run the plain path.
  if (target && target->id == HMC_T_LOGREG) c.impl = HMC_IMPL_PLAIN;
  if (target && target->id == HMC_T_CORR_GAUSS &&
      !(c.impl != HMC_IMPL_PLAIN && c.impl != HMC_IMPL_FUSED_SINGLE_CTA && hmc::gauss_fused_supported(*target)))
    c.impl = HMC_IMPL_PLAIN;
  hmc_ctx* ctx = nullptr;
  hmc_status st = hmc_create(target, num_chains * num_replicas, &c, cuda_stream, &ctx);
  if (st != HMC_OK) return st;
  ctx->K = num_replicas;
  ctx->outer_chains = num_chains;
  cudaError_t e = ctx_alloc(ctx, &ctx->betas, static_cast<size_t>(num_replicas));
  if (e == cudaSuccess) e = ctx_alloc(ctx, &ctx->swapped, static_cast<size_t>(num_chains * (num_replicas - 1)));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->betas, betas, sizeof(float) * num_replicas, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ctx->swapped, 0, static_cast<size_t>(num_chains * (num_replicas - 1)),
                        ctx->stream);
  if (e != cudaSuccess) {
    hmc_destroy(ctx);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? HMC_E_OOM : HMC_E_CUDA,
                std::string("replica set-up: ") + cudaGetErrorString(e));
  }
  *out = ctx;
  return HMC_OK;
}

hmc_status hmc_remc_swaps(const hmc_ctx* ctx, const uint8_t** swapped) {
  if (!ctx || !swapped || ctx->K < 2) return fail(nullptr, HMC_E_INVALID, "not a replica-exchange context");
  *swapped = ctx->swapped;
  return HMC_OK;
}

hmc_status hmc_synchronize(hmc_ctx* ctx) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  return check_device_flag(ctx);
}

hmc_status hmc_profile_dominant_kernel(hmc_ctx* ctx, int32_t sample_every) {
  if (!ctx) return fail(nullptr, HMC_E_INVALID, "ctx is NULL");
  if (sample_every < 0) return fail(ctx, HMC_E_INVALID, "sample_every must be >= 0");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "profile reset");
  // a captured graph holds the event records of the setting it was captured with
  if (sample_every != ctx->timer.every) drop_graph(ctx);
  ctx->timer.every = sample_every;
  ctx->timer.seen = 0;
  ctx->timer.recorded = 0;
  return HMC_OK;
}

hmc_status hmc_profile_read(hmc_ctx* ctx, double* avg_ms, uint64_t* samples, uint64_t* launches) {
  if (!ctx || !avg_ms || !samples || !launches) return fail(ctx, HMC_E_INVALID, "NULL argument");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "profile read");
  const uint64_t n = std::min<uint64_t>(ctx->timer.recorded, hmc::KernelTimer::kPairs);
  double total = 0.0;
  for (uint64_t k = 0; k < n; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ctx->timer.ev[2 * k], ctx->timer.ev[2 * k + 1]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event elapsed time");
    total += ms;
  }
  *avg_ms = n ? total / static_cast<double>(n) : 0.0;
  *samples = n;
  *launches = ctx->timer.seen;
  return HMC_OK;
}

hmc_status hmc_destroy(hmc_ctx* ctx) {
  if (!ctx) return HMC_OK;
  cudaStreamSynchronize(ctx->stream);
  ctx->timer.destroy();
  release(ctx);
  delete ctx;
  cudaGetLastError();   // teardown never leaves an error pending for the next call
  return HMC_OK;
}

const char* hmc_last_error(const hmc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_global_err.c_str();
}

int32_t hmc_uses_tensor_cores(const hmc_ctx* ctx) {
  return ctx && (ctx->use_tc || ctx->use_lrtc || ctx->use_lrgemm) ? 1 : 0;
}

hmc_status hmc_dominant_kernel_info(const hmc_ctx* ctx, char* name, int32_t name_len,
                                    int64_t* grad_evals_per_launch) {
  if (!ctx || !name || name_len < 1 || !grad_evals_per_launch)
    return fail(nullptr, HMC_E_INVALID, "NULL argument");
  const char* n = "";
  int64_t per = ctx->C;
  if (ctx->nuts_dense) {
    // a whole transition (leaf iterations of tile products + leaf kernel)
    n = "nuts_dense_transition";
  } else if (ctx->cfg.proposal == HMC_PROPOSAL_NUTS) {
    n = "k_nuts";          // leapfrog steps per launch vary: hmc_nuts_leapfrog_count
  } else if (ctx->use_tc && ctx->tc.fused && ctx->tc.pair) {
    n = "k_gauss_pair";
    per = ctx->C * ctx->cfg.num_leapfrog * ctx->dom_transitions;
  } else if (ctx->use_tc && ctx->tc.fused) {
    n = "k_gauss_fused";
    per = ctx->C * ctx->cfg.num_leapfrog;
  } else if (ctx->use_tc) {
    n = "k_gauss_tc_step";
  } else if (ctx->use_lrtc) {
    n = "k_lr_grad";
  } else if (ctx->use_lrgemm) {
    n = "k_gauss_tc_step<logreg>";   // both products of one gradient
  } else if (uses_fused_logreg(ctx)) {
    n = "k_logreg_fused";
    per = ctx->C * ctx->cfg.num_leapfrog;
  } else if (uses_fused_elementwise(ctx)) {
    n = "k_fused_elementwise";
    per = ctx->C * ctx->cfg.num_leapfrog;
  } else if (ctx->target.id == HMC_T_CORR_GAUSS) {
    n = "k_corr_gauss_grad";
  } else if (ctx->target.id == HMC_T_LOGREG) {
    n = "k_logreg_residual+k_logreg_grad_partial";
  } else if (ctx->target.id == HMC_T_FUNNEL) {
    n = "k_funnel_grad";
  } else {
    n = "k_std_normal_grad";
  }
  std::snprintf(name, static_cast<size_t>(name_len), "%s", n);
  *grad_evals_per_launch = per;
  return HMC_OK;
}

hmc_status hmc_grad_workspace_bytes(const hmc_target* target, int64_t num_chains, uint64_t* bytes) {
  std::string why;
  if (!bytes) return fail(nullptr, HMC_E_INVALID, "bytes is NULL");
  if (!valid_target(target, num_chains, &why)) return fail(nullptr, HMC_E_INVALID, why);
  *bytes = hmc::grad_workspace_bytes(*target, num_chains);
  return HMC_OK;
}

hmc_status hmc_target_log_prob_and_grad(const hmc_target* target, int64_t num_chains,
                                        const float* x, float* lp, float* grad, void* workspace,
                                        uint64_t workspace_bytes, void* cuda_stream) {
  std::string why;
  if (!valid_target(target, num_chains, &why)) return fail(nullptr, HMC_E_INVALID, why);
  if (!x || !lp || !grad) return fail(nullptr, HMC_E_INVALID, "x, lp and grad must be non-NULL");
  const size_t need = hmc::grad_workspace_bytes(*target, num_chains);
  if (need > workspace_bytes || (need && !workspace))
    return fail(nullptr, HMC_E_INVALID, "workspace smaller than hmc_grad_workspace_bytes");
  if (need && (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return fail(nullptr, HMC_E_INVALID, "workspace must be 256-byte aligned");
  cudaError_t e = hmc::launch_grad(*target, num_chains, x, lp, grad, workspace,
                                   static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "gradient launch");
  return HMC_OK;
}

hmc_status hmc_target_vjp_workspace_bytes(const hmc_target* target, int64_t num_chains,
                                          uint64_t* bytes) {
  uint64_t g = 0;
  hmc_status st = hmc_grad_workspace_bytes(target, num_chains, &g);
  if (st != HMC_OK) return st;
  *bytes = ((g + 255) & ~static_cast<uint64_t>(255)) + static_cast<uint64_t>(num_chains) * 4;
  return HMC_OK;
}

hmc_status hmc_target_vjp(const hmc_target* target, int64_t num_chains, const float* x,
                          const float* w, float* dx, void* workspace, uint64_t workspace_bytes,
                          void* cuda_stream) {
  uint64_t need = 0;
  hmc_status st = hmc_target_vjp_workspace_bytes(target, num_chains, &need);
  if (st != HMC_OK) return st;
  if (!x || !w || !dx) return fail(nullptr, HMC_E_INVALID, "x, w and dx must be non-NULL");
  if (!workspace || workspace_bytes < need)
    return fail(nullptr, HMC_E_INVALID, "workspace smaller than hmc_target_vjp_workspace_bytes");
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return fail(nullptr, HMC_E_INVALID, "workspace must be 256-byte aligned");
  const size_t gbytes = hmc::grad_workspace_bytes(*target, num_chains);
  char* base = static_cast<char*>(workspace);
  float* lp_tmp = reinterpret_cast<float*>(base + ((gbytes + 255) & ~static_cast<size_t>(255)));
  cudaError_t e = hmc::launch_vjp(*target, num_chains, x, w, dx, lp_tmp, base,
                                  static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "vjp launch");
  return HMC_OK;
}

hmc_status hmc_philox4x32_10(const uint32_t* counters, int64_t n, uint64_t seed, uint32_t* out,
                             void* cuda_stream) {
  if (n < 0 || (n > 0 && (!counters || !out)))
    return fail(nullptr, HMC_E_INVALID, "bad counters/out/n");
  cudaError_t e = hmc::launch_philox(counters, n, seed, out, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox launch");
  return HMC_OK;
}

hmc_status hmc_momentum(uint64_t seed, uint64_t t, int64_t num_chains, int32_t dim,
                        int64_t chain_offset, float* out, void* cuda_stream) {
  if (num_chains < 1 || num_chains > (1ll << 30) || dim < 1 || !out || chain_offset < 0 ||
      chain_offset + num_chains > (1ll << 32) || t > std::numeric_limits<uint32_t>::max())
    return fail(nullptr, HMC_E_INVALID, "bad momentum arguments");
  cudaError_t e = hmc::launch_momentum(seed, static_cast<uint32_t>(t), static_cast<int>(num_chains),
                                       dim, static_cast<uint32_t>(chain_offset), out,
                                       static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "momentum launch");
  return HMC_OK;
}

uint64_t hmc_kernel_launch_count(void) { return hmc::g_launches.load(); }

}  // extern "C"
