// Many posteriors of uneven dimension, data size and chain count sampled
// together (Section 2's premise -- independent chains, batched evaluation --
// applied across posteriors).  Two kinds of members:
//   grouped: every tile (8 chains) of every such posterior is a work item of
//     one persistent cooperative launch (k_batch_persistent) that runs all
//     their transitions: each CTA owns a fixed set of items, ordered by
//     estimated cost so the largest start first, and runs them transition by
//     transition.  A tile waits only after a transition that adapted its
//     posterior's step size, until the posterior's last tile has applied the
//     update (a per-posterior generation counter, bounded spin); transitions
//     with a fixed step size run without any barrier.  The bootstraps and
//     the launch are one CUDA graph.  Funnels, standard normals and small
//     logistic regressions (kGroupedMaxWork).
//   side: logistic regressions with longer data passes, sampled by their own
//     context (tensor-core products for dim <= 128, tiled SIMT products
//     otherwise) on a stream of their own, concurrently with the grouped graph.
// Each posterior keeps its own chain state, kernel results and
// dual-averaging scalar; a grouped posterior's adaptation reduction runs over
// its own tiles only, so every member's result equals sampling it alone.
#include <algorithm>
#include <cmath>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "elementwise_tile.cuh"
#include "hmc_device.cuh"
#include "hmc_internal.h"
#include "logreg_tile.cuh"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

struct BatchPost {
  int kind;            // hmc_target_id
  int nb;              // elementwise: Philox blocks per lane (1, 2, 4, 8)
  int ntiles;          // CTAs of this posterior
  int n_data;
  StepArgs s;          // C, D, L, seed, chain_offset, state and result pointers
  const float* X;
  const float* y;
  long long B, K;      // burn-in and kept transitions
  float* samples;      // [K x C x D] or null
  float* trace_eps;    // [K] or null
  uint8_t* trace_acc;  // [K x C] or null
};

template <int TARGET>
__device__ __forceinline__ bool elementwise_dispatch_r(const StepArgs& a, int nb, int tile, int ntiles,
                                                       bool reduce) {
  if (nb == 1) return elementwise_tile<TARGET, 1>(a, tile, ntiles, reduce);
  if (nb == 2) return elementwise_tile<TARGET, 2>(a, tile, ntiles, reduce);
  if (nb == 4) return elementwise_tile<TARGET, 4>(a, tile, ntiles, reduce);
  return elementwise_tile<TARGET, 8>(a, tile, ntiles, reduce);
}

constexpr unsigned long long kBatchWaitNs = 500000000ull;   // 0.5 s

// Every transition of every grouped posterior in one cooperative launch.
// Item (posterior, tile) i belongs to CTA i mod gridDim; each CTA runs its
// items for transition 0, then for transition 1, and so on.  Before
// transition t a tile of posterior p waits until gen[p] >= t when
// transition t - 1 adapted p's step size (the tile that applies an update
// sets gen[p] = t + 1 after it); the reduction itself runs on adapting
// transitions and on p's last, whose statistic the state reports, so the
// arithmetic is the per-transition launch's.  A CTA never waits on an item
// of a later transition than the one it runs, and all CTAs are resident, so
// every wait ends; each is bounded all the same (err, then the kernel
// returns).
__global__ void __launch_bounds__(256) k_batch_persistent(const BatchPost* __restrict__ posts,
                                                          const int2* __restrict__ items, int num_items,
                                                          uint32_t T, unsigned* gen, int* err) {
  __shared__ int abort_s;
  for (uint32_t t = 0; t < T; ++t) {
    for (int i = blockIdx.x; i < num_items; i += gridDim.x) {
      const int2 it = items[i];                            // (posterior, tile)
      const BatchPost& P = posts[it.x];
      const long long total = P.B + P.K;
      if (static_cast<long long>(t) >= total) continue;    // this posterior has finished
      const DAState* da = P.s.da;
      const bool adapt = da->adapt != 0;
      if (t > 0 && adapt && static_cast<long long>(t) - 1 < da->num_adapt) {
        if (threadIdx.x == 0) {
          abort_s = 0;
          const unsigned long long t0 = ptx::global_timer_ns();
          while (*reinterpret_cast<volatile unsigned*>(&gen[it.x]) < t) {
            if (ptx::global_timer_ns() - t0 > kBatchWaitNs) {
              atomicCAS(err, 0, 1);
              abort_s = 1;
              break;
            }
          }
          __threadfence();
        }
        __syncthreads();
        if (abort_s) return;
      }
      StepArgs a = P.s;
      a.t = t;
      a.t_full = t;
      const long long k = static_cast<long long>(t) - P.B;
      if (k >= 0) {
        a.sample_out = P.samples ? P.samples + k * static_cast<long long>(a.C) * a.D : nullptr;
        a.trace_acc = P.trace_acc ? P.trace_acc + k * a.C : nullptr;
        a.trace_eps = P.trace_eps ? P.trace_eps + k : nullptr;
      }
      const bool reduce = (adapt && static_cast<long long>(t) < da->num_adapt) ||
                          static_cast<long long>(t) == total - 1;
      bool updated;
      if (P.kind == HMC_T_LOGREG) {
        lr::LrArgs la{a, P.X, P.y, P.n_data};
        updated = lr::logreg_tile(la, it.y, P.ntiles, reduce);
      } else if (P.kind == HMC_T_FUNNEL) {
        updated = elementwise_dispatch_r<HMC_T_FUNNEL>(a, P.nb, it.y, P.ntiles, reduce);
      } else {
        updated = elementwise_dispatch_r<HMC_T_STD_NORMAL>(a, P.nb, it.y, P.ntiles, reduce);
      }
      if (updated && threadIdx.x == 0) {
        __threadfence();
        atomicExch(&gen[it.x], t + 1u);
      }
      __syncthreads();                                     // shared memory is the next item's
    }
  }
}

// A logistic regression joins the grouped launch when one gradient of all
// its chains is small (chains x rows x dim <= 2^22 multiply-adds); larger ones
// run their own context (tensor-core products where they apply) on a side
// stream, so that a grouped launch never waits on a long SIMT data pass.
constexpr int64_t kGroupedMaxWork = int64_t(1) << 22;

bool grouped_member(const hmc_target& t, int64_t C) {
  return t.id != HMC_T_LOGREG ||
         (logreg_fused_supported(t) && C * t.n_data * t.dim <= kGroupedMaxWork);
}

int blocks_per_lane(int D) {
  const int nblk = (D + 3) / 4;
  return nblk <= 32 ? 1 : nblk <= 64 ? 2 : nblk <= 128 ? 4 : 8;
}

}  // namespace
}  // namespace hmc

struct hmc_batch {
  int n = 0;
  cudaStream_t stream = nullptr;
  std::vector<hmc_ctx*> ctx;
  std::vector<hmc_target> targets;
  std::vector<int64_t> chains;
  std::vector<hmc::BatchPost> host_posts;   // grouped members only
  std::vector<int> member;                  // posterior -> index in host_posts, or -1 (side)
  std::vector<cudaStream_t> side_stream;    // per posterior (side members), else null
  std::vector<int> path;                    // per posterior: how it runs (hmc_batch_member_path)
  std::vector<double> ms_grouped, ms_tensor;   // the autotuner's measurements (NaN: not measured)
  std::vector<cudaEvent_t> side_done;
  cudaEvent_t fork = nullptr;
  hmc::BatchPost* dev_posts = nullptr;
  int2* dev_items = nullptr;
  int num_items = 0;
  unsigned* dev_gen = nullptr;   // per grouped posterior: transitions whose update is applied
  int* dev_err = nullptr;        // a bounded wait of the persistent launch gave up
  int grid = 0;                  // CTAs of the persistent launch (all resident)
  size_t smem = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<const void*> g_key;
  uint64_t g_launches = 0;
  std::string err;
};

namespace {

hmc_status bfail(hmc_batch* b, hmc_status st, const std::string& m) {
  if (b) b->err = m;
  else hmc::set_global_error(m);
  return st;
}

void batch_release(hmc_batch* b) {
  // contexts first: each synchronises its own stream, which may be a side stream
  for (hmc_ctx* c : b->ctx) hmc_destroy(c);
  b->ctx.clear();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaStream_t st : b->side_stream)
    if (st) cudaStreamDestroy(st);
  b->side_stream.clear();
  for (cudaEvent_t ev : b->side_done)
    if (ev) cudaEventDestroy(ev);
  b->side_done.clear();
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->dev_posts) cudaFree(b->dev_posts);
  if (b->dev_items) cudaFree(b->dev_items);
  if (b->dev_gen) cudaFree(b->dev_gen);
  if (b->dev_err) cudaFree(b->dev_err);
  b->dev_gen = nullptr;
  b->dev_err = nullptr;
  b->graph = nullptr;
  b->fork = nullptr;
  b->cap_stream = nullptr;
  b->dev_posts = nullptr;
  b->dev_items = nullptr;
  cudaGetLastError();   // release never leaves an error pending for the next call
}

// Rough cost of one tile transition: chains x leapfrog x per-gradient work.
double tile_cost(const hmc_target& t, const hmc_config& c) {
  const double per = t.id == HMC_T_LOGREG ? 2.0 * t.n_data * t.dim : 8.0 * t.dim;
  return per * c.num_leapfrog * 8.0;
}

// ---- autotuner ---------------------------------------------------------------
// A logistic regression can run as 8-chain shared-memory SIMT tiles in the
// grouped launch or on the tensor-core products (128-chain x 128-row pair
// tiles for dim <= 128, 128 x 64 one-CTA tiles otherwise) in a context of its
// own.  Which is faster depends on the shape; the autotuner times one
// transition of each path on the device (after one untimed) and keeps the
// answer per shape for the process.
enum { kPathGrouped = 0, kPathTensor = 1, kPathOwn = 2 };

struct TuneResult {
  int path;
  double ms_grouped, ms_tensor;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int>, TuneResult> g_tune_cache;

// Milliseconds per transition of `target` with C chains under `impl`, from
// a zero state with the configuration's step size held fixed; +inf if the
// context cannot be made.
double time_transition(const hmc_target& t, int64_t C, const hmc_config& base, int impl, cudaStream_t s) {
  hmc_config c = base;
  c.impl = impl;
  c.adapt = 0;
  c.num_adapt_steps = 0;
  c.use_graph = 0;
  c.max_transitions_per_launch = 0;
  const double inf = std::numeric_limits<double>::infinity();
  hmc_ctx* ctx = nullptr;
  if (hmc_create(&t, C, &c, s, &ctx) != HMC_OK) return inf;
  float* x = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double ms = inf;
  cudaError_t e = cudaMallocAsync(&x, sizeof(float) * C * t.dim, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(float) * C * t.dim, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess && hmc_bootstrap(ctx, x) == HMC_OK && hmc_step(ctx, x, 0, nullptr) == HMC_OK) {
    e = cudaEventRecord(e0, s);
    const bool ok = e == cudaSuccess && hmc_step(ctx, x, 1, nullptr) == HMC_OK;
    if (ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
      float f = 0.f;
      if (cudaEventElapsedTime(&f, e0, e1) == cudaSuccess) ms = f;
    }
  }
  if (hmc_synchronize(ctx) != HMC_OK) ms = inf;
  hmc_destroy(ctx);
  if (x) cudaFreeAsync(x, s);
  cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  return ms;
}

TuneResult tune_logreg(const hmc_target& t, int64_t C, const hmc_config& c, cudaStream_t s) {
  const auto key = std::make_tuple(t.dim, t.n_data, C, c.num_leapfrog);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  const double inf = std::numeric_limits<double>::infinity();
  // (SIMT tiles for a product past 2^31 multiply-adds would take seconds per
  // transition: the tensor cores win there without a measurement)
  const bool simt_ok = hmc::logreg_fused_supported(t) && C * t.n_data * t.dim <= (int64_t(1) << 31);
  const bool tensor_ok = hmc::logreg_tc_supported(t) || hmc::logreg_gemm_supported(t);
  TuneResult r{kPathGrouped, simt_ok ? time_transition(t, C, c, HMC_IMPL_FUSED_SIMT, s) : inf,
               tensor_ok ? time_transition(t, C, c, HMC_IMPL_FUSED_TENSOR, s) : inf};
  r.path = r.ms_tensor < r.ms_grouped ? kPathTensor : kPathGrouped;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = r;
  return r;
}

hmc_status batch_create(int32_t num_posteriors, const hmc_target* targets, const int64_t* num_chains,
                        const hmc_config* configs, void* cuda_stream, hmc_batch** out, bool autotune);

}  // namespace

extern "C" {

hmc_status hmc_batch_create(int32_t num_posteriors, const hmc_target* targets,
                            const int64_t* num_chains, const hmc_config* configs, void* cuda_stream,
                            hmc_batch** out) {
  return batch_create(num_posteriors, targets, num_chains, configs, cuda_stream, out, false);
}

hmc_status hmc_batch_create_autotuned(int32_t num_posteriors, const hmc_target* targets,
                                      const int64_t* num_chains, const hmc_config* configs,
                                      void* cuda_stream, hmc_batch** out) {
  return batch_create(num_posteriors, targets, num_chains, configs, cuda_stream, out, true);
}

hmc_status hmc_batch_member_path(const hmc_batch* b, int32_t i, int32_t* path, double* ms_grouped,
                                 double* ms_tensor) {
  if (!b || i < 0 || i >= b->n || !path) return bfail(nullptr, HMC_E_INVALID, "bad batch, index or path");
  *path = b->path[i];
  if (ms_grouped) *ms_grouped = b->ms_grouped[i];
  if (ms_tensor) *ms_tensor = b->ms_tensor[i];
  return HMC_OK;
}

}  // extern "C"

namespace {

hmc_status batch_create(int32_t num_posteriors, const hmc_target* targets, const int64_t* num_chains,
                        const hmc_config* configs, void* cuda_stream, hmc_batch** out, bool autotune) {
  if (!out) return bfail(nullptr, HMC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (num_posteriors < 1 || !targets || !num_chains || !configs)
    return bfail(nullptr, HMC_E_INVALID, "need >= 1 posterior and non-NULL arrays");
  hmc_batch* b = new hmc_batch();
  b->n = num_posteriors;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  std::vector<std::pair<double, int2>> items;
  for (int i = 0; i < num_posteriors; ++i) {
    const hmc_target& t = targets[i];
    if (t.id == HMC_T_CORR_GAUSS || (t.id == HMC_T_LOGREG && t.dim > hmc::lr::kLrMaxDim) ||
        ((t.id == HMC_T_FUNNEL || t.id == HMC_T_STD_NORMAL) && t.dim > hmc::kFusedElementwiseMaxDim)) {
      batch_release(b);
      delete b;
      return bfail(nullptr, HMC_E_UNSUPPORTED,
                   "batch posterior " + std::to_string(i) +
                       ": supported are LOGREG (dim <= 512), FUNNEL and STD_NORMAL (dim <= 1024)");
    }
    if (configs[i].proposal != HMC_PROPOSAL_LEAPFROG) {
      batch_release(b);
      delete b;
      return bfail(nullptr, HMC_E_UNSUPPORTED,
                   "batch posterior " + std::to_string(i) + ": batches run the leapfrog proposal only");
    }
    hmc_config c = configs[i];
    bool grouped = hmc::grouped_member(t, num_chains[i]);
    c.impl = HMC_IMPL_FUSED;       // side members: tensor-core products where they apply
    int path = grouped ? kPathGrouped : kPathOwn;
    double msg = std::nan(""), mst = std::nan("");
    if (autotune && t.id == HMC_T_LOGREG) {
      const TuneResult r = tune_logreg(t, num_chains[i], c, static_cast<cudaStream_t>(cuda_stream));
      path = r.path;
      msg = r.ms_grouped;
      mst = r.ms_tensor;
      grouped = path == kPathGrouped;
      c.impl = grouped ? HMC_IMPL_FUSED_SIMT : HMC_IMPL_FUSED_TENSOR;
    }
    b->path.push_back(path);
    b->ms_grouped.push_back(msg);
    b->ms_tensor.push_back(mst);
    // side members replay their own graph: enqueueing thousands of launches
    // eagerly would fill the launch queue and serialise the side streams
    c.use_graph = grouped ? 0 : 1;
    cudaStream_t side = nullptr;
    cudaEvent_t done = nullptr;
    if (!grouped) {
      if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        delete b;
        return bfail(nullptr, HMC_E_CUDA, "side stream creation failed");
      }
    }
    b->side_stream.push_back(side);
    b->side_done.push_back(done);
    hmc_ctx* ctx = nullptr;
    hmc_status st = hmc_create(&t, num_chains[i], &c, grouped ? cuda_stream : side, &ctx);
    if (st != HMC_OK) {
      const std::string m = "batch posterior " + std::to_string(i) + ": " + hmc_last_error(nullptr);
      batch_release(b);
      delete b;
      return bfail(nullptr, st, m);
    }
    b->ctx.push_back(ctx);
    b->targets.push_back(t);
    b->chains.push_back(num_chains[i]);
    if (!grouped) {
      b->member.push_back(-1);
      continue;
    }
    hmc::BatchPost P{};
    P.kind = t.id;
    P.nb = hmc::blocks_per_lane(t.dim);
    P.ntiles = static_cast<int>((num_chains[i] + 7) / 8);     // 8 chains per tile for every kind
    P.n_data = static_cast<int>(t.n_data);
    P.X = t.X;
    P.y = t.y;
    b->member.push_back(static_cast<int>(b->host_posts.size()));
    b->host_posts.push_back(P);
    const double cost = tile_cost(t, c);
    const int gi = b->member.back();
    for (int tile = 0; tile < P.ntiles; ++tile) items.push_back({cost, make_int2(gi, tile)});
    if (t.id == HMC_T_LOGREG) b->smem = std::max(b->smem, hmc::lr::logreg_smem_bytes(t.dim));
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const auto& a, const auto& c) { return a.first > c.first; });
  std::vector<int2> flat;
  for (auto& it : items) flat.push_back(it.second);
  b->num_items = static_cast<int>(flat.size());
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !b->host_posts.empty())
    e = cudaMalloc(&b->dev_posts, sizeof(hmc::BatchPost) * b->host_posts.size());
  if (e == cudaSuccess && !flat.empty()) e = cudaMalloc(&b->dev_items, sizeof(int2) * flat.size());
  if (e == cudaSuccess && !flat.empty())
    e = cudaMemcpy(b->dev_items, flat.data(), sizeof(int2) * flat.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->host_posts.empty())
    e = cudaMalloc(&b->dev_gen, sizeof(unsigned) * b->host_posts.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->dev_err, 0, sizeof(int));
  // the attribute belongs to the kernel, not to this batch: set the maximum
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(hmc::k_batch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(hmc::lr::logreg_smem_bytes(hmc::lr::kLrMaxDim)));
  // the persistent launch takes as many CTAs as can be resident at once
  if (e == cudaSuccess && b->num_items > 0) {
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hmc::k_batch_persistent, 256, b->smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    b->grid = std::min(b->num_items, sms * per_sm);
  }
  if (e != cudaSuccess) {
    const hmc_status st = e == cudaErrorMemoryAllocation ? HMC_E_OOM : HMC_E_CUDA;
    cudaGetLastError();
    batch_release(b);
    delete b;
    return bfail(nullptr, st, std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  *out = b;
  return HMC_OK;
}

}  // namespace

extern "C" {

hmc_status hmc_batch_sample_chain(hmc_batch* b, float* const* x_inout, const int64_t* num_burnin,
                                  const int64_t* num_results, float* const* samples_out,
                                  float* const* trace_step_size, uint8_t* const* trace_accept) {
  if (!b) return bfail(nullptr, HMC_E_INVALID, "batch is NULL");
  if (!x_inout || !num_burnin || !num_results)
    return bfail(b, HMC_E_INVALID, "x_inout, num_burnin and num_results must be non-NULL");
  long long T = 0;
  std::vector<const void*> key;
  for (int i = 0; i < b->n; ++i) {
    if (!x_inout[i]) return bfail(b, HMC_E_INVALID, "x_inout[" + std::to_string(i) + "] is NULL");
    if (num_burnin[i] < 0 || num_results[i] < 0) return bfail(b, HMC_E_INVALID, "negative step count");
    if (num_burnin[i] + num_results[i] > 0xFFFFFFFFll)
      return bfail(b, HMC_E_INVALID, "too many transitions");
    if (b->member[i] < 0) continue;
    T = std::max<long long>(T, num_burnin[i] + num_results[i]);
    hmc::BatchPost& P = b->host_posts[b->member[i]];
    P.B = num_burnin[i];
    P.K = num_results[i];
    P.samples = samples_out ? samples_out[i] : nullptr;
    P.trace_eps = trace_step_size ? trace_step_size[i] : nullptr;
    P.trace_acc = trace_accept ? trace_accept[i] : nullptr;
    key.insert(key.end(), {x_inout[i], P.samples, P.trace_eps, P.trace_acc,
                           reinterpret_cast<const void*>(P.B), reinterpret_cast<const void*>(P.K)});
  }
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, std::string("fork: ") + cudaGetErrorString(e));
  // side members: their own streams, concurrent with the grouped graph
  for (int i = 0; i < b->n; ++i) {
    if (b->member[i] >= 0) continue;
    e = cudaStreamWaitEvent(b->side_stream[i], b->fork, 0);
    if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, std::string("side wait: ") + cudaGetErrorString(e));
    hmc_status st = hmc_sample_chain(b->ctx[i], x_inout[i], num_burnin[i], num_results[i],
                                     samples_out ? samples_out[i] : nullptr,
                                     trace_step_size ? trace_step_size[i] : nullptr,
                                     trace_accept ? trace_accept[i] : nullptr);
    if (st != HMC_OK)
      return bfail(b, st, "side posterior " + std::to_string(i) + ": " + hmc_last_error(b->ctx[i]));
    e = cudaEventRecord(b->side_done[i], b->side_stream[i]);
    if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, std::string("side record: ") + cudaGetErrorString(e));
  }
  if (!b->host_posts.empty()) {
    const bool hit = b->graph && key == b->g_key;
    if (!hit) {
      if (b->graph) cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      if (!b->cap_stream) {
        e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, cudaGetErrorString(e));
      }
      for (int i = 0; i < b->n; ++i)
        if (b->member[i] >= 0) b->host_posts[b->member[i]].s = hmc::ctx_step_args(b->ctx[i], x_inout[i], 0);
      const uint64_t l0 = hmc::g_launches.load();
      e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess)
        return bfail(b, HMC_E_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
      hmc_status st = HMC_OK;
      e = cudaMemcpyAsync(b->dev_posts, b->host_posts.data(),
                          sizeof(hmc::BatchPost) * b->host_posts.size(), cudaMemcpyHostToDevice,
                          b->cap_stream);
      for (int i = 0; i < b->n && st == HMC_OK && e == cudaSuccess; ++i)
        if (b->member[i] >= 0) st = hmc::ctx_bootstrap_on(b->ctx[i], x_inout[i], b->cap_stream);
      if (st == HMC_OK && e == cudaSuccess)
        e = cudaMemsetAsync(b->dev_gen, 0, sizeof(unsigned) * b->host_posts.size(), b->cap_stream);
      if (st == HMC_OK && e == cudaSuccess && T > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(b->grid));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = b->smem;
        cfg.stream = b->cap_stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, hmc::k_batch_persistent, static_cast<const hmc::BatchPost*>(b->dev_posts),
                               static_cast<const int2*>(b->dev_items), b->num_items, static_cast<uint32_t>(T),
                               b->dev_gen, b->dev_err);
        hmc::count_launch();
        if (e == cudaSuccess) e = cudaGetLastError();
      }
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
      if (st != HMC_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st != HMC_OK) return bfail(b, st, "bootstrap failed");
        return bfail(b, HMC_E_CUDA, std::string("batch capture: ") +
                                        cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return bfail(b, HMC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      b->g_launches = hmc::g_launches.load() - l0;
      hmc::g_launches.fetch_sub(b->g_launches);
      b->g_key = key;
    }
    e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    hmc::count_launch(b->g_launches);
  }
  // join: the caller's stream waits for every side member
  for (int i = 0; i < b->n; ++i) {
    if (b->member[i] >= 0) continue;
    e = cudaStreamWaitEvent(b->stream, b->side_done[i], 0);
    if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, std::string("join: ") + cudaGetErrorString(e));
  }
  return HMC_OK;
}

hmc_status hmc_batch_synchronize(hmc_batch* b) {
  if (!b) return bfail(nullptr, HMC_E_INVALID, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  int flag = 0;
  if (e == cudaSuccess && b->dev_err) e = cudaMemcpy(&flag, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(b, HMC_E_CUDA, std::string("batch synchronize: ") + cudaGetErrorString(e));
  if (flag) return bfail(b, HMC_E_TIMEOUT, "a bounded wait of the grouped launch gave up");
  for (int i = 0; i < b->n; ++i) {
    hmc_status st = hmc_synchronize(b->ctx[i]);
    if (st != HMC_OK) return bfail(b, st, "posterior " + std::to_string(i) + ": " + hmc_last_error(b->ctx[i]));
  }
  return HMC_OK;
}

hmc_status hmc_batch_destroy(hmc_batch* b) {
  if (!b) return HMC_OK;
  cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
  return HMC_OK;
}

const char* hmc_batch_last_error(const hmc_batch* b) { return b ? b->err.c_str() : ""; }

hmc_ctx* hmc_batch_context(hmc_batch* b, int32_t i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->ctx[i];
}

}  // extern "C"
