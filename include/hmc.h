/*
 * libhmc: vectorised multi-chain Hamiltonian Monte Carlo on one GB300 GPU.
 *
 * The method is the HMC transition kernel and sample_chain driver of
 * "tfp.mcmc: Modern Markov Chain Monte Carlo Tools Built for Modern Hardware"
 * (Lao et al., 2020): thousands of independent chains advance in lockstep
 * (Section 2, "Pervasive Data Parallelism"); each transition draws one
 * momentum per state variable per chain, runs a fixed number of leapfrog steps
 * with the step size broadcast over the state, and accepts or rejects every
 * chain by Metropolis-Hastings with a per-chain select (Section 2.1).  A
 * transition consumes and produces (state, kernel results) of fixed structure,
 * and the kernel results cache the target log-prob and gradient of the
 * accepted state (Section 4.1, one_step / bootstrap_results).  The driver runs
 * burn-in transitions whose states are not stored, then kept ones, and traces
 * kernel-result fields (Section 4.2).  Step-size adaptation during burn-in
 * (Section 4.1, the step-size adaptation wrapper) uses dual averaging
 * (Hoffman and Gelman 2014, Algorithm 5).
 *
 * Conventions for every call:
 *   - Pointers named "device" are CUDA device pointers owned by the caller
 *     unless stated otherwise.  State arrays are row-major [chains x dim]
 *     float32 (chain c's state is x[c*dim .. c*dim+dim-1]).
 *   - All work is enqueued asynchronously on the stream given to hmc_create
 *     (or to the call); nothing synchronises unless stated.
 *   - Every call returns an hmc_status; nothing throws or aborts.  The text of
 *     the last error of a context is available from hmc_last_error.
 *   - Results depend only on (seed, chain index + chain_offset, transition
 *     index) and the chain's own state: never on the number of chains or on
 *     the other chains in the batch (Section 2's batch semantics).
 */
#ifndef HMC_H_
#define HMC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMC_OK = 0,
  HMC_E_INVALID = 1,      /* bad argument: NULL pointer, size, step size, id */
  HMC_E_OOM = 2,          /* device workspace allocation failed */
  HMC_E_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  HMC_E_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  HMC_E_UNSUPPORTED = 5   /* valid request the library does not implement */
} hmc_status;

/* Target families.  Log-densities are up to an additive constant.
 *   STD_NORMAL  log p = -|x|^2/2 (the worked example of Section 1, any dim)
 *   CORR_GAUSS  log p = -x^T P x / 2, P symmetric positive definite [dim x dim]
 *   LOGREG      Bayesian logistic regression, prior N(0, I):
 *               log p = sum_i y_i z_i - softplus(z_i) - |x|^2/2, z = X x,
 *               X [n_data x dim] row-major, y [n_data] in {0, 1}
 *   FUNNEL      Neal's funnel, state (v, x_1..x_{dim-1}): v ~ N(0, 9),
 *               x_i | v ~ N(0, e^v); dim >= 2 */
typedef enum {
  HMC_T_STD_NORMAL = 0,
  HMC_T_CORR_GAUSS = 1,
  HMC_T_LOGREG = 2,
  HMC_T_FUNNEL = 3
} hmc_target_id;

/* Target description.  P, X, y are device pointers owned by the caller; they
 * are read, never written, and must stay valid until the context that uses
 * them is destroyed.  Unused pointers may be NULL. */
typedef struct {
  int32_t id;          /* hmc_target_id */
  int32_t dim;         /* state dimension D >= 1 */
  int64_t n_data;      /* LOGREG: rows of X; otherwise 0 */
  const float* P;      /* CORR_GAUSS: [dim x dim] */
  const float* X;      /* LOGREG: [n_data x dim] */
  const float* y;      /* LOGREG: [n_data] */
} hmc_target;

typedef enum {
  HMC_IMPL_FUSED = 0,             /* fused transition kernels (default); dense
                                     Gaussians run on CTA pairs (cta_group::2) */
  HMC_IMPL_PLAIN = 1,             /* one kernel launch per operation per
                                     leapfrog step */
  HMC_IMPL_FUSED_SINGLE_CTA = 2,  /* as FUSED, but the dense-Gaussian
                                     transition on single CTAs (32 chains,
                                     each CTA streaming P by TMA) */
  HMC_IMPL_FUSED_TENSOR = 3,      /* as FUSED, but a logistic regression
                                     always takes the tensor-core products
                                     (whatever its size) */
  HMC_IMPL_FUSED_SIMT = 4         /* as FUSED, but a logistic regression
                                     always takes the shared-memory SIMT
                                     transition (dim <= 512; 8 chains per
                                     CTA tile) */
} hmc_impl;

/* Inner (uncalibrated) kernel of the Metropolis-Hastings composition,
 * Section 4.1's MetropolisHastings(Uncalibrated...(...)). */
typedef enum {
  HMC_PROPOSAL_LEAPFROG = 0,     /* Hamiltonian: num_leapfrog leapfrog steps from a
                                    fresh momentum; with num_leapfrog = 1 this is
                                    the Langevin (MALA) proposal x + eps^2/2 grad
                                    + eps z with its exact correction */
  HMC_PROPOSAL_RANDOM_WALK = 1,  /* x' = x + eps z, z ~ N(0, I) (the momentum
                                    stream), log alpha = log p(x') - log p(x);
                                    num_leapfrog is ignored; runs the plain
                                    one-launch-per-operation path */
  HMC_PROPOSAL_NUTS = 2          /* the No-U-Turn Sampler (Section 2.3) with the
                                    recursion unrolled: num_leapfrog is the
                                    maximum tree depth (1..10, at most 2^depth - 1
                                    leapfrog steps per transition); dim <= 512,
                                    for CORR_GAUSS a multiple of 4
                                    (HMC_E_UNSUPPORTED otherwise).  STD_NORMAL
                                    and FUNNEL: one warp per chain, each chain's
                                    tree independent; CORR_GAUSS and LOGREG: the
                                    chains advance in lockstep, one leaf per
                                    iteration (tensor-core gradient products of
                                    the chains still building, then one leaf
                                    kernel), the iterations a conditional node
                                    of a CUDA graph: a call that enqueues
                                    transitions on a stream that is not
                                    capturing captures them on the context's
                                    private stream and launches the graph; the
                                    impl field is ignored; the step size
                                    adapts to the mean over a tree's leaves of
                                    min(1, exp(H0 - H)); is_accepted reports
                                    whether the state moved, log_accept_ratio
                                    the log of that mean */
} hmc_proposal_kind;

/* Sampler configuration (the HamiltonianMonteCarlo constructor arguments of
 * the Section 1 listing plus adaptation). */
typedef struct {
  int32_t num_leapfrog;     /* L >= 1 */
  float step_size;          /* initial (or fixed) step size, finite, > 0 */
  uint64_t seed;            /* Philox key */
  int32_t adapt;            /* 0: fixed step size; 1: dual averaging */
  float target_accept;      /* dual-averaging target in (0, 1) */
  int64_t num_adapt_steps;  /* transitions t < num_adapt_steps adapt (>= 0) */
  int32_t impl;             /* hmc_impl */
  int64_t chain_offset;     /* chain c draws the random streams of chain
                               c + chain_offset */
  int32_t use_graph;        /* 1: hmc_sample_chain captures bootstrap and all
                               transitions as one CUDA graph on first use and
                               replays it while its pointer and count
                               arguments stay the same; 0: plain launches */
  int32_t max_transitions_per_launch;
                            /* dense Gaussian on CTA pairs: hmc_sample_chain
                               runs at most this many transitions per kernel
                               launch (>= 0; 0: no limit, the whole chain in
                               one cooperative launch; 1: one launch per
                               transition, e.g. for a profiler that cannot
                               replay cooperative cluster launches) */
  int32_t proposal;         /* hmc_proposal_kind: the inner kernel of the
                               Metropolis-Hastings composition (Section 4.1) */
} hmc_config;

/* Kernel results of the last transition.  All pointers are device pointers
 * owned by the context, valid until the next call on it or hmc_destroy. */
typedef struct {
  const float* target_log_prob;   /* [chains] log p of the current state */
  const float* grad;              /* [chains x dim] its gradient */
  const uint8_t* is_accepted;     /* [chains] 1 if the proposal was accepted */
  const float* log_accept_ratio;  /* [chains] H_0 - H_L, -inf if non-finite */
  const float* step_size;         /* [1] step size the NEXT transition uses */
} hmc_kernel_results;

typedef struct hmc_ctx hmc_ctx;

/* Create a sampler context for `num_chains` chains of `target`, enqueuing on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).  Validates the
 * arguments (HMC_E_INVALID) and allocates the context's device workspace
 * (HMC_E_OOM); it does not touch the chain state.  On success *out owns the
 * workspace until hmc_destroy.  Sections 3.1 and 4.1. */
hmc_status hmc_create(const hmc_target* target, int64_t num_chains, const hmc_config* config,
                      void* cuda_stream, hmc_ctx** out);

/* Device memory accounting (no counterpart in the paper; for admission by
 * memory budget, as a sampling server does).
 *   hmc_create_device_bytes: bytes hmc_create would request from the device
 *     for these arguments (its workspace: kernel results, scratch of the
 *     path the configuration selects), without creating anything; the
 *     target's data pointers may be NULL.  HMC_E_INVALID on bad sizes or
 *     configuration.
 *   hmc_context_device_bytes: bytes a context holds now -- what
 *     hmc_create allocated, plus what later calls added (the batch-means
 *     buffers of hmc_sample_chain_streaming_ess, the staging buffers of
 *     hmc_sample_chain_host).  Neither counts the caller's own buffers (state,
 *     samples, target data). */
hmc_status hmc_create_device_bytes(const hmc_target* target, int64_t num_chains, const hmc_config* config,
                                   uint64_t* bytes);
hmc_status hmc_context_device_bytes(const hmc_ctx* ctx, uint64_t* bytes);

/* bootstrap_results (Section 4.1): evaluate log p and its gradient at x0
 * ([chains x dim], device, read only) into the context's kernel results and
 * reset the step size and the dual-averaging state to the configuration's. */
hmc_status hmc_bootstrap(hmc_ctx* ctx, const float* x0);

/* one_step (Sections 3.1, 4.1): advance every chain by one HMC transition
 * with transition index t (which keys the random streams and, when adapting,
 * decides whether this transition adapts).  x_inout [chains x dim] (device)
 * must hold the state that the kernel results belong to (the one passed to
 * hmc_bootstrap or returned by the previous step); it is overwritten with the
 * next state.  If `out` is not NULL it receives the kernel results. */
hmc_status hmc_step(hmc_ctx* ctx, float* x_inout, uint64_t t, hmc_kernel_results* out);

/* sample_chain (Section 4.2): bootstrap at x_inout, run num_burnin + num_results
 * transitions with t = 0, 1, ..., keep the state after each of the last
 * num_results transitions, and leave the final state in x_inout.
 *   samples_out     [num_results x chains x dim] device or NULL
 *   trace_step_size [num_results] device or NULL: step size each kept
 *                   transition used
 *   trace_accept    [num_results x chains] device or NULL: is_accepted
 * Both counts must be >= 0. */
hmc_status hmc_sample_chain(hmc_ctx* ctx, float* x_inout, int64_t num_burnin, int64_t num_results,
                            float* samples_out, float* trace_step_size, uint8_t* trace_accept);

/* The streaming-expectations driver the paper plans (Section 4.2: for state
 * too large to store a full trace): same transitions as hmc_sample_chain, but
 * instead of storing kept states it updates, after every kept transition,
 * Welford running moments per chain and dimension (device, [chains x dim],
 * caller-owned): mean_out = mean of the kept states, m2_out = sum of squared
 * deviations from it (variance = m2 / (num_results - 1)).  Both are left
 * unwritten when num_results == 0.  Traces as in hmc_sample_chain. */
hmc_status hmc_sample_chain_streaming(hmc_ctx* ctx, float* x_inout, int64_t num_burnin,
                                      int64_t num_results, float* mean_out, float* m2_out,
                                      float* trace_step_size, uint8_t* trace_accept);

/* The streaming driver with batch-means effective sample sizes (Section
 * 4.2's trace-free driver; the estimator is the replicated batch means of
 * Gupta and Vats 2020, batch means after Geyer 1992): as
 * hmc_sample_chain_streaming, and the kept draws of every chain are also cut
 * into nb = num_results / batch_size consecutive batches of batch_size draws
 * (a last partial batch is left out of the batch means).  ess_out (device,
 * [dim], caller-owned) receives, per dimension,
 *   chains x num_results x W / V,
 * W = mean over chains of m2 / (num_results - 1) (the sample variance),
 * V = batch_size x the sum over all chains' batches of (batch mean - grand
 * mean of the batch means)^2 / (chains x nb - 1).  batch_size = num_results
 * (one batch per chain) makes V the spread of the chain means across chains,
 * which also sees autocorrelation longer than any batch.  A dimension whose
 * batch means never vary gets +inf (NaN if nothing varies).  Needs
 * batch_size >= 1, nb >= 1 and chains x nb >= 2 (else HMC_E_INVALID);
 * replica sets (hmc_remc_create) are HMC_E_UNSUPPORTED.  The context
 * allocates 3 x chains x dim floats of workspace on first use. */
hmc_status hmc_sample_chain_streaming_ess(hmc_ctx* ctx, float* x_inout, int64_t num_burnin,
                                          int64_t num_results, int64_t batch_size, float* mean_out,
                                          float* m2_out, float* ess_out, float* trace_step_size,
                                          uint8_t* trace_accept);

/* Same as hmc_sample_chain with every argument in HOST memory (x_inout,
 * samples_out, trace buffers; pinned or pageable).  Copies the initial state
 * to the device, samples, copies the results back and synchronises the
 * context's stream before returning.  When samples_out is pinned and holds
 * at least 512 MiB, the kept samples are copied back in segments (at most
 * 16, each at least 256 MiB, each split over four copy streams) while the
 * later transitions run (replica sets included; not under NUTS); the
 * results are the same. */
hmc_status hmc_sample_chain_host(hmc_ctx* ctx, float* x_inout, int64_t num_burnin,
                                 int64_t num_results, float* samples_out,
                                 float* trace_step_size, uint8_t* trace_accept);

/* sample_chain in pieces (Section 4.2's driver, split for checkpointing):
 * run transitions t_begin .. t_end - 1 of a chain with num_burnin burn-in
 * transitions, so that consecutive calls [0, k), [k, n) give exactly the
 * chain of one hmc_sample_chain(num_burnin, n - num_burnin) call.  With
 * t_begin == 0 the chain is bootstrapped at x_inout; otherwise x_inout
 * (device) and the context's kernel results and adaptation state must hold
 * the state after transition t_begin - 1 (left there by the previous call,
 * or put there by hmc_restore_state: HMC_E_INVALID if neither happened).
 * Kept transitions t >= num_burnin write output index
 * t - max(num_burnin, t_begin) of samples_out [.. x chains x dim],
 * trace_step_size and trace_accept (device, each may be NULL).  No CUDA
 * graph is captured. */
hmc_status hmc_sample_chain_range(hmc_ctx* ctx, float* x_inout, int64_t num_burnin, int64_t t_begin,
                                  int64_t t_end, float* samples_out, float* trace_step_size,
                                  uint8_t* trace_accept);

/* Checkpoint and resume (no counterpart in the paper; the paper's kernels
 * are pure functions of (state, kernel results), Section 4.1, which is what
 * makes this possible).  A context's resumable state is its kernel results
 * (the cached log p [chains] and gradient [chains x dim] of the current
 * state) and its dual-averaging state; the chain state itself is the
 * caller's x.
 *   hmc_state_bytes: size of that state in bytes.
 *   hmc_save_state: copy it to host memory `out` (at least that many bytes)
 *     after the context's pending work; synchronises; HMC_E_TIMEOUT if a
 *     device-side wait gave up.
 *   hmc_restore_state: load it into a context created with the same target
 *     (family and dim), chain count, replica count and configuration --
 *     typically a fresh one in another process -- after which
 *     hmc_sample_chain_range / hmc_step continue the saved chain bit for bit;
 *     HMC_E_INVALID if the saved state belongs to another target, chain count
 *     or build.  Synchronous. */
hmc_status hmc_state_bytes(const hmc_ctx* ctx, uint64_t* bytes);
hmc_status hmc_save_state(hmc_ctx* ctx, void* out, uint64_t bytes);
hmc_status hmc_restore_state(hmc_ctx* ctx, const void* in, uint64_t bytes);

/* Test support (no counterpart in the paper): for every later launch of the
 * dense-Gaussian CTA-pair kernel, the time after which its grid barrier (the
 * dual-averaging meeting point of a multi-transition launch) gives up, in
 * nanoseconds (default 500000000), and a barrier generation (1, 2, ...; 0:
 * none) that can never complete, so that a test can make the bounded wait
 * run out: the kernel then skips its remaining transitions and returns, and
 * hmc_synchronize reports HMC_E_TIMEOUT.  Process-wide. */
void hmc_debug_set_grid_barrier(uint64_t wait_limit_ns, int32_t unreachable_generation);

/* Copy the current dual-averaging state to host memory and synchronise:
 * out[0] = step size of the next transition, out[1] = log eps_bar,
 * out[2] = h_bar, out[3] = adaptation steps taken, out[4] = last transition's
 * acceptance statistic (mean over chains of min(1, alpha)). */
hmc_status hmc_read_adaptation(hmc_ctx* ctx, double out[5]);

/* Wait for the context's stream; HMC_E_TIMEOUT if a device-side bounded
 * wait gave up since the context was created (the kernel that gave up
 * skipped its writes; the state is then not meaningful). */
hmc_status hmc_synchronize(hmc_ctx* ctx);

/* 1 if the context's transitions run the tensor-core (tcgen05, 3xTF32)
 * kernels: CORR_GAUSS with dim % 4 == 0 under HMC_IMPL_FUSED; LOGREG under
 * HMC_IMPL_FUSED_TENSOR, or under HMC_IMPL_FUSED with n_data > 2048, chains x
 * n_data x dim > 2^22, or fewer than (SMs / 2) x 8 chains and n_data x dim
 * > 10^4 (CTA pairs for dim <= 128, one-CTA tile products otherwise); NUTS
 * on either dense target.  0 otherwise. */
int32_t hmc_uses_tensor_cores(const hmc_ctx* ctx);

/* Measurement support (no counterpart in the paper): the name of the kernel
 * hmc_profile_dominant_kernel times for this context and how many chain
 * gradient evaluations one launch of it performs (chains x leapfrog steps for
 * the one-launch-per-transition kernels, times the transitions of the last
 * hmc_sample_chain where one launch ran all of them -- the dense Gaussian on
 * CTA pairs -- and chains for one gradient product). */
hmc_status hmc_dominant_kernel_info(const hmc_ctx* ctx, char* name, int32_t name_len,
                                    int64_t* grad_evals_per_launch);

/* Measurement support (no counterpart in the paper): time one launch in
 * every `sample_every` of the context's dominant kernel -- the fused
 * transition kernel, or the target-gradient product(s) of the plain path --
 * with CUDA events on the context's stream.  0 disables.  Synchronises the
 * stream and resets the counters.  A sample_chain graph records the events
 * of the setting it was captured with: changing sample_every drops the graph
 * (the next hmc_sample_chain captures again); calling again with the same
 * value only resets the counters. */
hmc_status hmc_profile_dominant_kernel(hmc_ctx* ctx, int32_t sample_every);

/* Average duration (ms) of the timed launches since the last reset, how many
 * were timed (at most 2048, the most recent ones) and how many dominant
 * launches occurred.  Synchronises the context's stream. */
hmc_status hmc_profile_read(hmc_ctx* ctx, double* avg_ms, uint64_t* samples, uint64_t* launches);

/* Total leapfrog steps (= gradient evaluations) of the NUTS transitions run
 * on this context since it was created (their number varies per chain and
 * transition).  Synchronises the context's stream.  HMC_E_INVALID if the
 * context does not run NUTS. */
hmc_status hmc_nuts_leapfrog_count(hmc_ctx* ctx, uint64_t* out);

/* NUTS: the leaf steps on the schedule's critical path since the context was
 * created.  Dense targets (CORR_GAUSS, LOGREG): the lockstep loop's
 * iterations, one batched gradient of the chains still building their trees
 * each (hmc_nuts_leapfrog_count / (iterations x num_chains) is the fraction
 * of chain rows that did useful work).  STD_NORMAL, FUNNEL: the sum over
 * launches of the longest chain's leaf count in the launch, the serial work
 * no launch can finish before.  Synchronises the context's stream.
 * HMC_E_INVALID if the context does not run NUTS. */
hmc_status hmc_nuts_leaf_iterations(hmc_ctx* ctx, uint64_t* out);

/* The composition's two halves as separate calls (Section 4.1:
 * MetropolisHastings wrapping an uncalibrated kernel).  hmc_step is exactly
 * hmc_propose followed by hmc_mh_select with the same t (bit-identical
 * results).  Both need a context created with impl = HMC_IMPL_PLAIN (or
 * proposal = HMC_PROPOSAL_RANDOM_WALK) and no replicas; otherwise
 * HMC_E_UNSUPPORTED.  hmc_bootstrap must come first (HMC_E_INVALID).
 *
 * hmc_propose: draws transition t's proposal from the state x ([chains x
 * dim], device, read only) and its cached log p / gradient, without
 * accepting it.  *out receives device pointers owned by the context, valid
 * until the next call on it: the proposed state, its log p and gradient, and
 * log alpha per chain (-inf where non-finite). */
typedef struct {
  const float* x;                 /* [chains x dim] proposed state */
  const float* target_log_prob;   /* [chains] */
  const float* grad;              /* [chains x dim] */
  const float* log_accept_ratio;  /* [chains] */
} hmc_proposal;

hmc_status hmc_propose(hmc_ctx* ctx, const float* x, uint64_t t, hmc_proposal* out);

/* The Metropolis-Hastings step for the last hmc_propose (which must have used
 * the same t and state): chain c takes the proposal iff log u < log alpha
 * (u from transition t's accept stream), x_inout and the cached log p /
 * gradient are updated in place, the step size adapts as in hmc_step, and
 * *out (may be NULL) is filled as by hmc_step. */
hmc_status hmc_mh_select(hmc_ctx* ctx, float* x_inout, uint64_t t, hmc_kernel_results* out);

/* Release the context's workspace.  NULL is accepted. */
hmc_status hmc_destroy(hmc_ctx* ctx);

/* Text of the last error on `ctx` ("" if none); with ctx == NULL, the last
 * error of a call that had no context (e.g. a failed hmc_create).  The string
 * is owned by the library and valid until the next call on the same context. */
const char* hmc_last_error(const hmc_ctx* ctx);

/* ---- Replica exchange ----------------------------------------------------
 * Replica exchange Monte Carlo (Section 2.2): every chain carries K replicas
 * whose target log-probabilities are scaled by inverse temperatures
 * betas[k] (betas[0] = 1 is the distribution of interest); the replicas are
 * one more batch axis -- replica k of chain c is row c * K + k of the
 * [chains * K x dim] state -- so every replica advances by the ordinary HMC
 * transition (its own random streams, those of row c * K + k), and after the
 * transition with index t adjacent replicas (k, k + 1) with k = t % 2,
 * t % 2 + 2, ... swap their states iff
 *   log u < (betas[k] - betas[k+1]) (log p(x_{k+1}) - log p(x_k)),
 * u from the counter generator at (k, c, t, tag 2).  Kept samples are taken
 * after the exchange.  The context's log-prob and gradient results are the
 * tempered ones.  Fixed step size only (adapt = 0; HMC_E_UNSUPPORTED
 * otherwise); chain_offset must be 0.  Dense targets (CORR_GAUSS, LOGREG)
 * use the one-launch-per-operation path; the others the fused kernels.
 * betas: host array of num_replicas values in (0, 1].  All other calls
 * (hmc_bootstrap, hmc_step, hmc_sample_chain, ...) take the
 * [num_chains * num_replicas x dim] state. */
hmc_status hmc_remc_create(const hmc_target* target, int64_t num_chains, int32_t num_replicas,
                           const float* betas, const hmc_config* config, void* cuda_stream,
                           hmc_ctx** out);

/* Device pointer to the last exchange step's outcomes, [num_chains x
 * (num_replicas - 1)] uint8 (1 = pair (k, k+1) swapped; 0 also for pairs not
 * proposed at that step), owned by the context. */
hmc_status hmc_remc_swaps(const hmc_ctx* ctx, const uint8_t** swapped);

/* ---- Batches of posteriors ------------------------------------------------
 * Many posteriors of uneven dimension, data size and chain count sampled
 * together (the independent-chain batching of Section 2 applied across
 * posteriors).  Funnels, standard normals and small logistic regressions
 * (chains x rows x dim <= 2^22) share one persistent kernel launch for all
 * their transitions (one tile per 8 chains, largest tiles first; a tile waits
 * only for its own posterior's step-size update after a transition that
 * adapts it), with the bootstraps as one CUDA graph; larger logistic regressions run their own transitions
 * (tensor-core products for dim <= 128) on streams of their own,
 * concurrently.  Each posterior keeps
 * its own state, kernel results and dual-averaging step size, so its result
 * equals sampling it alone.  Supported families: LOGREG (dim <= 512), FUNNEL
 * and STD_NORMAL (dim <= 1024); others give HMC_E_UNSUPPORTED.  All work is
 * ordered after prior work on the batch's stream and the stream waits for
 * all of it. */
typedef struct hmc_batch hmc_batch;

/* Create a batch of num_posteriors posteriors: targets[i], num_chains[i] and
 * configs[i] as for hmc_create (impl and use_graph are ignored).  Allocates
 * each posterior's workspace; errors as hmc_create, text via
 * hmc_last_error(NULL). */
hmc_status hmc_batch_create(int32_t num_posteriors, const hmc_target* targets,
                            const int64_t* num_chains, const hmc_config* configs, void* cuda_stream,
                            hmc_batch** out);

/* As hmc_batch_create, with each logistic regression's execution path
 * chosen by measurement (an autotuner; no counterpart in the paper): the
 * grouped launch's 8-chain shared-memory SIMT tiles, or the tensor-core
 * products in a context of its own (128-chain x 128-row tiles on CTA pairs
 * for dim <= 128, 128 x 64 one-CTA tiles otherwise).  One
 * transition of each path is timed on the device (after one untimed) from a
 * zero state with the configured step size fixed, and the faster is taken;
 * the answer is kept per shape (dim, rows, chains, leapfrog steps) for the
 * life of the process, so later batches of the same shapes pay no
 * measurement.  The timing runs on cuda_stream and synchronises it.  A
 * member's result equals sampling it alone with impl HMC_IMPL_FUSED_SIMT
 * (grouped) or HMC_IMPL_FUSED_TENSOR (tensor cores). */
hmc_status hmc_batch_create_autotuned(int32_t num_posteriors, const hmc_target* targets,
                                      const int64_t* num_chains, const hmc_config* configs,
                                      void* cuda_stream, hmc_batch** out);

/* How posterior i of a batch runs: *path = 0 in the grouped launch, 1 in a
 * context of its own on the tensor-core products (autotuned), 2 in a context
 * of its own on the path HMC_IMPL_FUSED selects (the untuned rule).  With the
 * autotuner, ms_grouped / ms_tensor (each may be NULL) receive the measured
 * milliseconds per transition of the two paths (+inf where a path does not
 * apply; NaN for members the tuner did not measure). */
hmc_status hmc_batch_member_path(const hmc_batch* batch, int32_t i, int32_t* path, double* ms_grouped,
                                 double* ms_tensor);

/* sample_chain (Section 4.2) for every posterior at once: arrays of
 * num_posteriors entries, entry i as in hmc_sample_chain for posterior i
 * (x_inout[i] device [C_i x D_i]; samples_out / trace arrays may be NULL, and
 * so may their entries).  Posteriors with fewer transitions stop early.  The
 * first call with a given set of pointers and counts captures the loop as a
 * graph; later calls replay it. */
hmc_status hmc_batch_sample_chain(hmc_batch* batch, float* const* x_inout,
                                  const int64_t* num_burnin, const int64_t* num_results,
                                  float* const* samples_out, float* const* trace_step_size,
                                  uint8_t* const* trace_accept);

/* The context of posterior i (owned by the batch; for hmc_read_adaptation
 * and hmc_synchronize).  NULL if i is out of range. */
hmc_ctx* hmc_batch_context(hmc_batch* batch, int32_t i);

/* Wait for all of the batch's work; HMC_E_TIMEOUT if a bounded device-side
 * wait gave up (the grouped launch's per-posterior adaptation barrier, or a
 * posterior context's own). */
hmc_status hmc_batch_synchronize(hmc_batch* batch);

/* Text of the batch's last error ("" if none). */
const char* hmc_batch_last_error(const hmc_batch* batch);

/* Release the batch and every posterior's workspace.  NULL is accepted. */
hmc_status hmc_batch_destroy(hmc_batch* batch);

/* Bytes of device scratch that hmc_target_log_prob_and_grad needs for
 * `num_chains` chains of `target` (0 for targets that need none; LOGREG needs
 * the C x N residual matrix and split-K partial sums).  Returns 0 and sets
 * *bytes on success, HMC_E_INVALID on a bad target or count. */
hmc_status hmc_grad_workspace_bytes(const hmc_target* target, int64_t num_chains, uint64_t* bytes);

/* Target log-prob and gradient for `num_chains` states x [chains x dim]
 * (device) into lp [chains] and grad [chains x dim] (device, caller-owned),
 * enqueued on `cuda_stream`.  This is the batched target evaluation of
 * Section 2.1 ("list of vectors", one row per chain) and the adjoint used by
 * the autograd binding: the vector-Jacobian product of log p with upstream
 * weights w is w_c * grad[c].  `workspace` is caller-owned device scratch of
 * at least hmc_grad_workspace_bytes bytes, 256-byte aligned (may be NULL when
 * that size is 0).  Allocates nothing.  Returns HMC_E_INVALID on bad sizes,
 * pointers or a too-small workspace. */
hmc_status hmc_target_log_prob_and_grad(const hmc_target* target, int64_t num_chains,
                                        const float* x, float* lp, float* grad,
                                        void* workspace, uint64_t workspace_bytes,
                                        void* cuda_stream);

/* Workspace for hmc_target_vjp: the gradient's scratch plus one float per
 * chain. */
hmc_status hmc_target_vjp_workspace_bytes(const hmc_target* target, int64_t num_chains,
                                          uint64_t* bytes);

/* Vector-Jacobian product of the batched log-density (the adjoint behind the
 * autograd binding; the paper obtains gradients by automatic differentiation,
 * Section 3 and its footnote on TF autodiff): dx[c, :] = w[c] * grad log p(x_c)
 * for x, dx [chains x dim] and w [chains] (device, caller-owned).  The forward
 * pass is recomputed, nothing from it is stored.  `workspace` (device,
 * 256-byte aligned, >= hmc_target_vjp_workspace_bytes) is caller-owned.
 * HMC_E_INVALID on bad sizes, pointers or workspace. */
hmc_status hmc_target_vjp(const hmc_target* target, int64_t num_chains, const float* x,
                          const float* w, float* dx, void* workspace, uint64_t workspace_bytes,
                          void* cuda_stream);

/* Same as hmc_target_log_prob_and_grad, for callers that cannot allocate
 * device memory at all (no counterpart in the paper).  Some callers must not
 * call cudaMalloc when they evaluate a gradient: a host process that owns the
 * whole device-memory budget (e.g. a sampling server that reserves HBM up
 * front for every admitted job's resident chain state), or a latency-critical
 * loop where cudaMalloc's implicit synchronisation would stall other streams.
 * This entry point takes its scratch from a fixed 64 MiB array inside the
 * library's device image (held on every GPU that loads the library until the
 * process exits) and calls no allocating routine.  The caller passes inputs
 * and outputs only, as in hmc_target_log_prob_and_grad.
 *   - The first call on a device resolves the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     The address is cached for the device's primary context: after
 *     cudaDeviceReset (which destroys that context and unloads the module)
 *     the cached address is stale, so do not call this entry point again in
 *     a process that has reset the device.
 *   - Requests needing more scratch than 64 MiB (LOGREG with a large
 *     chains x n_data) return HMC_E_INVALID with the sizes in the error text.
 *   - All calls share the one array and it keeps the last call's contents;
 *     nothing in it must start at zero, but calls whose kernels overlap on
 *     the GPU race on it: serialise them (one stream, or events). */
hmc_status hmc_target_log_prob_and_grad_noalloc(const hmc_target* target, int64_t num_chains,
                                                const float* x, float* lp, float* grad,
                                                void* cuda_stream);

/* The counter-based generator behind every random draw (the paper names
 * none; this is Philox4x32-10 of Salmon, Moraes, Dror and Shaw, SC'11):
 * out[4i..4i+3] = Philox4x32-10(counters[4i..4i+3], key = (seed lo32,
 * seed hi32)) for i < n.  counters and out are device arrays of 4n uint32.
 * Exposed so that callers can check the stream bit for bit. */
hmc_status hmc_philox4x32_10(const uint32_t* counters, int64_t n, uint64_t seed, uint32_t* out,
                             void* cuda_stream);

/* The momentum draw of one transition (Section 2.1: one independent N(0,1)
 * momentum per state variable per chain): out [chains x dim] (device) for
 * chains chain_offset .. chain_offset + num_chains - 1 at transition t. */
hmc_status hmc_momentum(uint64_t seed, uint64_t t, int64_t num_chains, int32_t dim,
                        int64_t chain_offset, float* out, void* cuda_stream);

/* Number of kernels this library launched in the calling process so far
 * (a host-side counter, for launch accounting). */
uint64_t hmc_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HMC_H_ */
