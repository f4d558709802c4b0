// HMC transition kernels (Section 2.1): momentum draw, leapfrog, energy,
// Metropolis-Hastings select and the dual-averaging update.
//
// Fused path for targets whose gradient is elementwise plus row reductions
// (standard normal, funnel): one warp per chain keeps x, p and g of its chain
// in registers for all L leapfrog steps and the accept test, so one
// transition is one launch that reads x, g once and writes them once.
//
// Plain path (any target): one launch per operation per leapfrog step --
// begin (momentum + H_0), kick-drift, gradient, kick, ..., accept -- the
// shape a framework that evaluates a batched target op by op produces.
#include <cmath>

#include "elementwise_tile.cuh"
#include "hmc_device.cuh"
#include "hmc_internal.h"

namespace hmc {

unsigned accept_blocks(int C) { return static_cast<unsigned>((C + 7) / 8); }

namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ void finish_block(const StepArgs& a, float prob, bool has_chain) {
  accept_block_finish<kWarpsPerBlock>(a.da, a.partials, prob, has_chain, a.C, a.t_full);
}

// ------------------------------------------------------ fused elementwise --
template <int TARGET, int NB>
__global__ void __launch_bounds__(256) k_fused_elementwise(StepArgs a) {
  elementwise_tile<TARGET, NB>(a, static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
}

// ------------------------------------------------------------ plain path --
// p ~ N(0, I); xp = x; gp = g; h0 = -lp + |p|^2/2   (warp per chain)
__global__ void k_plain_begin(StepArgs a, PlainBuffers b) {
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.C) return;
  const int D = a.D;
  const int64_t row = static_cast<int64_t>(c) * D;
  const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
  float kin = 0.f;
  for (int j = lane; 4 * j < D; j += 32) {
    const float4 z = momentum4(a.seed, static_cast<uint32_t>(j), chain, a.t);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int i = 0; i < 4 && 4 * j + i < D; ++i) {
      const int64_t e = row + 4 * j + i;
      b.p[e] = zz[i];
      b.xp[e] = a.x[e];
      b.gp[e] = a.g[e];
      kin = fmaf(zz[i], zz[i], kin);
    }
  }
  kin = warp_sum(kin);
  if (lane == 0) b.h0[c] = -a.lp[c] + 0.5f * kin;
}

// p += eps/2 gp; xp += eps p
__global__ void k_plain_kick_drift(int64_t n, float* __restrict__ p, const float* __restrict__ gp,
                                   float* __restrict__ xp, const DAState* __restrict__ da) {
  const float eps = da->eps;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float pi = fmaf(0.5f * eps, gp[i], p[i]);
    p[i] = pi;
    xp[i] = fmaf(eps, pi, xp[i]);
  }
}

// p += eps/2 gp
__global__ void k_plain_kick(int64_t n, float* __restrict__ p, const float* __restrict__ gp,
                             const DAState* __restrict__ da) {
  const float eps = da->eps;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = fmaf(0.5f * eps, gp[i], p[i]);
}

// Random-walk proposal (Section 4.1's composition with a symmetric inner
// kernel): xp = x + eps z with z the transition's momentum draws; p = 0, so
// the energies below reduce to log alpha = log p(xp) - log p(x).
__global__ void k_rw_begin(StepArgs a, PlainBuffers b) {
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.C) return;
  const int D = a.D;
  const int64_t row = static_cast<int64_t>(c) * D;
  const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
  const float eps = a.da->eps;
  for (int j = lane; 4 * j < D; j += 32) {
    const float4 z = momentum4(a.seed, static_cast<uint32_t>(j), chain, a.t);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int i = 0; i < 4 && 4 * j + i < D; ++i) {
      const int64_t e = row + 4 * j + i;
      b.p[e] = 0.f;
      b.xp[e] = fmaf(eps, zz[i], a.x[e]);
    }
  }
  if (lane == 0) b.h0[c] = -a.lp[c];
}

// log alpha = H_0 - H_L of chain c (warp per chain; every lane gets it)
__device__ __forceinline__ float plain_log_alpha(const StepArgs& a, const PlainBuffers& b, int c,
                                                 int lane) {
  const int D = a.D;
  const int64_t row = static_cast<int64_t>(c) * D;
  float kin = 0.f;
  for (int d = lane; d < D; d += 32) kin = fmaf(b.p[row + d], b.p[row + d], kin);
  kin = 0.5f * warp_sum(kin);
  const float h1 = -b.lpp[c] + kin;
  float la = b.h0[c] - h1;
  if (!isfinite(la)) la = -INFINITY;
  return la;
}

// Metropolis-Hastings select of chain c given log alpha; returns min(1, alpha)
__device__ __forceinline__ float plain_select(const StepArgs& a, const PlainBuffers& b, int c, int lane,
                                              float la) {
  const int D = a.D;
  const int64_t row = static_cast<int64_t>(c) * D;
  const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
  int acc = 0;
  if (lane == 0) acc = accept_log_uniform(a.seed, chain, a.t) < la;
  acc = __shfl_sync(0xffffffffu, acc, 0);
  for (int d = lane; d < D; d += 32) {
    if (acc) {
      a.x[row + d] = b.xp[row + d];
      a.g[row + d] = b.gp[row + d];
    }
    if (a.sample_out) a.sample_out[row + d] = a.x[row + d];
  }
  if (lane == 0) {
    if (acc) a.lp[c] = b.lpp[c];
    a.is_accepted[c] = static_cast<uint8_t>(acc);
    a.log_accept[c] = la;
    if (a.trace_acc) a.trace_acc[c] = static_cast<uint8_t>(acc);
    if (c == 0 && a.trace_eps) a.trace_eps[0] = a.da->eps;
  }
  return accept_prob(la);
}

// H_L, log alpha, Metropolis-Hastings select, traces, dual averaging
__global__ void k_plain_accept(StepArgs a, PlainBuffers b) {
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) prob = plain_select(a, b, c, lane, plain_log_alpha(a, b, c, lane));
  finish_block(a, prob, has_chain);
}

// the split: log alpha only ...
__global__ void k_plain_ratio(StepArgs a, PlainBuffers b) {
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.C) return;
  const float la = plain_log_alpha(a, b, c, lane);
  if (lane == 0) b.la[c] = la;
}

// ... then the select from it
__global__ void k_plain_select(StepArgs a, PlainBuffers b) {
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) prob = plain_select(a, b, c, lane, b.la[c]);
  finish_block(a, prob, has_chain);
}

__global__ void k_da_init(DAState* da, float eps0, int adapt, float delta, long long num_adapt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  da->log_eps = log(static_cast<double>(eps0));
  da->log_eps_bar = 0.0;
  da->h_bar = 0.0;
  da->mu = log(10.0 * static_cast<double>(eps0));
  da->delta = static_cast<double>(delta);
  da->last_stat = 0.0;
  da->m = 0;
  da->num_adapt = num_adapt;
  da->eps = eps0;
  da->adapt = adapt;
  da->arrive = 0u;
}

__global__ void k_philox_words(const uint32_t* __restrict__ ctr, int64_t n, uint64_t seed,
                               uint32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 w = philox(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
  }
}

// one thread per (chain, Philox block)
__global__ void k_momentum(uint64_t seed, uint32_t t, int C, int D, uint32_t chain_offset,
                           float* __restrict__ out) {
  const int nblk = (D + 3) / 4;
  const int64_t total = static_cast<int64_t>(C) * nblk;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(i / nblk), j = static_cast<int>(i % nblk);
    const float4 z = momentum4(seed, static_cast<uint32_t>(j), static_cast<uint32_t>(c) + chain_offset, t);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int k = 0; k < 4 && 4 * j + k < D; ++k) out[static_cast<int64_t>(c) * D + 4 * j + k] = zz[k];
  }
}


template <int TARGET, int NB>
void launch_fe(const StepArgs& a, cudaStream_t s) {
  k_fused_elementwise<TARGET, NB><<<accept_blocks(a.C), 256, 0, s>>>(a);
}

template <int TARGET>
void launch_fe_dim(const StepArgs& a, cudaStream_t s) {
  const int nblk = (a.D + 3) / 4;           // Philox blocks per chain
  if (nblk <= 32) launch_fe<TARGET, 1>(a, s);
  else if (nblk <= 64) launch_fe<TARGET, 2>(a, s);
  else if (nblk <= 128) launch_fe<TARGET, 4>(a, s);
  else launch_fe<TARGET, 8>(a, s);
}

inline unsigned elementwise_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<unsigned>(std::min<int64_t>(b, 152 * 16));
}

}  // namespace

cudaError_t launch_fused_elementwise(int target_id, const StepArgs& a, cudaStream_t s,
                                     KernelTimer* timer) {
  if (a.D > kFusedElementwiseMaxDim) return cudaErrorInvalidValue;
  if (target_id != HMC_T_STD_NORMAL && target_id != HMC_T_FUNNEL) return cudaErrorInvalidValue;
  if (timer) timer->begin(s);
  if (target_id == HMC_T_STD_NORMAL) launch_fe_dim<HMC_T_STD_NORMAL>(a, s);
  else launch_fe_dim<HMC_T_FUNNEL>(a, s);
  if (timer) timer->end(s);
  count_launch();
  return cudaGetLastError();
}

// the proposal: leapfrog trajectory (HMC; MALA at L = 1) or random walk
static cudaError_t plain_proposal(const hmc_target& t, const StepArgs& a, const PlainBuffers& b,
                                  void* grad_ws, cudaStream_t s, KernelTimer* timer) {
  const int64_t n = static_cast<int64_t>(a.C) * a.D;
  if (a.proposal == HMC_PROPOSAL_RANDOM_WALK) {
    k_rw_begin<<<accept_blocks(a.C), 256, 0, s>>>(a, b);
    count_launch();
    cudaError_t e = launch_grad(t, a.C, b.xp, b.lpp, b.gp, grad_ws, s, timer);
    if (e == cudaSuccess && a.K > 1) e = launch_temper(a.C, a.D, b.lpp, b.gp, a.betas, a.K, s);
    return e;
  }
  k_plain_begin<<<accept_blocks(a.C), 256, 0, s>>>(a, b);
  count_launch();
  for (int l = 0; l < a.L; ++l) {
    k_plain_kick_drift<<<elementwise_blocks(n), 256, 0, s>>>(n, b.p, b.gp, b.xp, a.da);
    count_launch();
    cudaError_t e = launch_grad(t, a.C, b.xp, b.lpp, b.gp, grad_ws, s, timer);
    if (e == cudaSuccess && a.K > 1) e = launch_temper(a.C, a.D, b.lpp, b.gp, a.betas, a.K, s);
    if (e != cudaSuccess) return e;
    k_plain_kick<<<elementwise_blocks(n), 256, 0, s>>>(n, b.p, b.gp, a.da);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_plain_transition(const hmc_target& t, const StepArgs& a, const PlainBuffers& b,
                                    void* grad_ws, cudaStream_t s, KernelTimer* timer) {
  cudaError_t e = plain_proposal(t, a, b, grad_ws, s, timer);
  if (e != cudaSuccess) return e;
  k_plain_accept<<<accept_blocks(a.C), 256, 0, s>>>(a, b);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_plain_propose(const hmc_target& t, const StepArgs& a, const PlainBuffers& b,
                                 void* grad_ws, cudaStream_t s) {
  cudaError_t e = plain_proposal(t, a, b, grad_ws, s, nullptr);
  if (e != cudaSuccess) return e;
  k_plain_ratio<<<accept_blocks(a.C), 256, 0, s>>>(a, b);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_plain_select(const StepArgs& a, const PlainBuffers& b, cudaStream_t s) {
  k_plain_select<<<accept_blocks(a.C), 256, 0, s>>>(a, b);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_philox_words<<<elementwise_blocks(n), 256, 0, s>>>(ctr, n, seed, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_momentum(uint64_t seed, uint32_t t, int C, int D, uint32_t chain_offset,
                            float* out, cudaStream_t s) {
  k_momentum<<<elementwise_blocks(static_cast<int64_t>(C) * ((D + 3) / 4)), 256, 0, s>>>(
      seed, t, C, D, chain_offset, out);
  count_launch();
  return cudaGetLastError();
}

// The streaming driver's moment update after kept draw k, one element per
// thread (welford_update).
__global__ void k_welford(int64_t n, const float* __restrict__ x, int64_t k, WelfordOut w) {
  const WelfordCoef q = welford_coef(k, w.bsize);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    welford_update(w, q, k, i, x[i]);
}

cudaError_t launch_welford(int64_t n, const float* x, int64_t k, float* mean, float* m2,
                           int64_t bsize, float* bsum, float* bmean, float* bm2, cudaStream_t s) {
  k_welford<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 152 * 16)), 256, 0, s>>>(
      n, x, k, WelfordOut{mean, m2, bsize, bsum, bmean, bm2});
  count_launch();
  return cudaGetLastError();
}

// Replicated batch-means effective sample size per dimension: the C nb
// batch means pooled about their grand mean (per chain, bmean / bm2 are the
// Welford mean and sum of squared deviations of its nb batch means), so
// SS = sum_c [bm2_c + nb (bmean_c - grand)^2] with grand = mean_c bmean_c,
// and ess[d] = C K (sum_c m2_c / (C (K - 1))) / (bsize SS / (C nb - 1)).  A
// block covers 32 dimensions (one per lane, coalesced rows) with its 8 warps
// striding over chains in two passes (grand mean, then sums); float64.
__global__ void __launch_bounds__(256) k_bm_ess(int64_t C, int D, int64_t K, int64_t bsize,
                                                const float* __restrict__ m2,
                                                const float* __restrict__ bmean,
                                                const float* __restrict__ bm2, float* __restrict__ ess) {
  __shared__ double a_s[8][32], b_s[8][32];
  __shared__ double grand_s[32];
  const int d = blockIdx.x * 32 + threadIdx.x;
  const double nb = static_cast<double>(K / bsize);
  double sb = 0.0;
  if (d < D)
    for (int64_t c = threadIdx.y; c < C; c += 8) sb += static_cast<double>(bmean[c * D + d]);
  a_s[threadIdx.y][threadIdx.x] = sb;
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int y = 1; y < 8; ++y) sb += a_s[y][threadIdx.x];
    grand_s[threadIdx.x] = sb / static_cast<double>(C);
  }
  __syncthreads();
  const double grand = grand_s[threadIdx.x];
  double w = 0.0, ss = 0.0;
  if (d < D)
    for (int64_t c = threadIdx.y; c < C; c += 8) {
      const double dev = static_cast<double>(bmean[c * D + d]) - grand;
      w += static_cast<double>(m2[c * D + d]);
      ss += static_cast<double>(bm2[c * D + d]) + nb * dev * dev;
    }
  __syncthreads();
  a_s[threadIdx.y][threadIdx.x] = w;
  b_s[threadIdx.y][threadIdx.x] = ss;
  __syncthreads();
  if (threadIdx.y == 0 && d < D) {
    for (int y = 1; y < 8; ++y) {
      w += a_s[y][threadIdx.x];
      ss += b_s[y][threadIdx.x];
    }
    const double Cd = static_cast<double>(C), Kd = static_cast<double>(K);
    const double W = w / (Cd * (Kd - 1.0));
    const double sig2 = static_cast<double>(bsize) * ss / (Cd * nb - 1.0);
    ess[d] = static_cast<float>(Cd * Kd * W / sig2);
  }
}

cudaError_t launch_bm_ess(int64_t C, int D, int64_t K, int64_t bsize, const float* m2, const float* bmean,
                          const float* bm2, float* ess, cudaStream_t s) {
  k_bm_ess<<<static_cast<unsigned>((D + 31) / 32), dim3(32, 8), 0, s>>>(C, D, K, bsize, m2, bmean, bm2,
                                                                        ess);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_temper(int64_t rows, int D, float* __restrict__ lp, float* __restrict__ g,
                         const float* __restrict__ betas, int K) {
  const int64_t n = rows * D;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / D;
    const float beta = betas[r % K];
    g[i] *= beta;
    if (i % D == 0) lp[r] *= beta;
  }
}

cudaError_t launch_temper(int64_t rows, int D, float* lp, float* g, const float* betas, int K,
                          cudaStream_t s) {
  const int64_t n = rows * D;
  k_temper<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 152 * 16)), 256, 0, s>>>(
      rows, D, lp, g, betas, K);
  count_launch();
  return cudaGetLastError();
}

// Replica exchange (Section 2.2): for chain c and pair (k, k+1), k = t % 2,
// t % 2 + 2, ..., swap the two replicas' states iff
// log u < (beta_k - beta_{k+1}) (log p(x_{k+1}) - log p(x_k)), with u drawn from
// the counter generator at (k, c, t, tag 2).  Cached log p and gradient are
// tempered: the untempered values are lp / beta and g / beta.  Warp per pair.
__global__ void k_remc_swap(int64_t chains, int K, int D, float* __restrict__ x,
                            float* __restrict__ lp, float* __restrict__ g,
                            const float* __restrict__ betas, uint64_t seed, uint32_t t,
                            uint8_t* __restrict__ swapped) {
  const int npairs = K - 1;
  const int64_t w = blockIdx.x * static_cast<int64_t>(kWarpsPerBlock) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= chains * npairs) return;
  const int64_t c = w / npairs;
  const int k = static_cast<int>(w % npairs);
  if ((k & 1) != static_cast<int>(t & 1u)) {
    if (lane == 0) swapped[w] = 0;
    return;
  }
  const int64_t r0 = c * K + k, r1 = r0 + 1;
  const float b0 = betas[k], b1 = betas[k + 1];
  float raw0, raw1;
  int sw = remc_swap_accept(lp[r0], lp[r1], b0, b1, seed, static_cast<uint32_t>(k), static_cast<uint32_t>(c),
                            t, &raw0, &raw1);
  sw = __shfl_sync(0xffffffffu, sw, 0);
  if (sw) {
    for (int d = lane; d < D; d += 32) {
      const int64_t e0 = r0 * D + d, e1 = r1 * D + d;
      const float xa = x[e0], xb = x[e1];
      x[e0] = xb;
      x[e1] = xa;
      const float ga = g[e0], gb = g[e1];
      g[e0] = gb / b1 * b0;
      g[e1] = ga / b0 * b1;
    }
    if (lane == 0) {
      lp[r0] = b0 * raw1;
      lp[r1] = b1 * raw0;
    }
  }
  if (lane == 0) swapped[w] = static_cast<uint8_t>(sw);
}

cudaError_t launch_remc_swap(int64_t chains, int K, int D, float* x, float* lp, float* g,
                             const float* betas, uint64_t seed, uint32_t t, uint8_t* swapped,
                             cudaStream_t s) {
  const int64_t warps = chains * (K - 1);
  k_remc_swap<<<static_cast<unsigned>((warps + kWarpsPerBlock - 1) / kWarpsPerBlock),
                32 * kWarpsPerBlock, 0, s>>>(chains, K, D, x, lp, g, betas, seed, t, swapped);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_da_init(DAState* da, float eps0, int adapt, float delta, long long num_adapt,
                           cudaStream_t s) {
  k_da_init<<<1, 32, 0, s>>>(da, eps0, adapt, delta, num_adapt);
  count_launch();
  return cudaGetLastError();
}

}  // namespace hmc
