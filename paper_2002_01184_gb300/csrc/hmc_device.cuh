// Device-side building blocks shared by the CUDA kernels of libhmc:
// the counter-based generator, Box-Muller, warp reductions and the
// dual-averaging state.  Host code never includes the kernels' arithmetic
// from anywhere else.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hmc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11).  The paper draws "one
// independent momentum per state variable per chain" (Section 2.1) but names
// no generator; a counter-based one needs no state in HBM and makes every
// draw a pure function of (seed, chain, transition, stream tag).
//   key     = (seed lo32, seed hi32)
//   counter = (block j, chain c, transition t, tag s)
//   tag 0 -> momentum, words 4j..4j+3 feed state dims 4j..4j+3
//   tag 1 -> Metropolis-Hastings uniform (word 0 of block 0)
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kTagMomentum = 0u;
constexpr uint32_t kTagAccept = 1u;

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
    const uint32_t lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// (w + 1/2) * 2^-32 in float32: strictly positive, at most 1.
__device__ __forceinline__ float word_to_uniform(uint32_t w) {
  return fmaf(static_cast<float>(w), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// log((w + 1/2) 2^-32) to float32 relative accuracy for every word: below
// 1/2 the uniform itself is accurate; above, 1 - u = (~w + 1/2) 2^-32 is
// formed exactly from the complement and log1p avoids the cancellation that
// rounding u to float32 would cause next to 1.
__device__ __forceinline__ float log_word_uniform(uint32_t w) {
  if (w < 0x80000000u) return logf(word_to_uniform(w));
  return log1pf(-word_to_uniform(~w));
}

// Box-Muller: r = sqrt(-2 log u_a), (r cos 2 pi u_b, r sin 2 pi u_b).
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
  const float r = sqrtf(-2.0f * log_word_uniform(wa));
  float s, c;
  sincospif(2.0f * word_to_uniform(wb), &s, &c);
  return make_float2(r * c, r * s);
}

// Four normals for state dims 4j..4j+3 of chain `chain` at transition t.
__device__ __forceinline__ float4 momentum4(uint64_t seed, uint32_t j, uint32_t chain, uint32_t t) {
  const uint4 w = philox(make_uint4(j, chain, t, kTagMomentum),
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  const float2 a = box_muller(w.x, w.y);
  const float2 b = box_muller(w.z, w.w);
  return make_float4(a.x, a.y, b.x, b.y);
}

// The normal for state dim d alone (component d % 4 of momentum4(d / 4)):
// one Box-Muller pair instead of two.
__device__ __forceinline__ float momentum1(uint64_t seed, uint32_t d, uint32_t chain, uint32_t t) {
  const uint4 w = philox(make_uint4(d >> 2, chain, t, kTagMomentum),
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  const float2 z = (d & 2u) ? box_muller(w.z, w.w) : box_muller(w.x, w.y);
  return (d & 1u) ? z.y : z.x;
}

__device__ __forceinline__ float accept_log_uniform(uint64_t seed, uint32_t chain, uint32_t t) {
  const uint4 w = philox(make_uint4(0u, chain, t, kTagAccept),
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  return log_word_uniform(w.x);
}

// Replica exchange (Section 2.2) after transition t: replicas k and k + 1 of
// outer chain c, with tempered log-densities lp0 = b0 log p(x0) and
// lp1 = b1 log p(x1), swap iff log u < (b0 - b1) (log p(x1) - log p(x0)), u
// from counter (k, c, t, 2).  raw0 / raw1 receive log p(x0) / log p(x1).
// Every kernel that exchanges replicas decides through this function, so
// they agree bit for bit.
__device__ __forceinline__ bool remc_swap_accept(float lp0, float lp1, float b0, float b1, uint64_t seed,
                                                 uint32_t k, uint32_t c, uint32_t t, float* raw0,
                                                 float* raw1) {
  *raw0 = lp0 / b0;
  *raw1 = lp1 / b1;
  const float la = (b0 - b1) * (*raw1 - *raw0);
  const uint4 u = philox(make_uint4(k, c, t, 2u), static_cast<uint32_t>(seed),
                         static_cast<uint32_t>(seed >> 32));
  return log_word_uniform(u.x) < la;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// min(1, exp(log_alpha)); a non-finite ratio counts as 0 (a divergence).
__device__ __forceinline__ float accept_prob(float log_alpha) {
  return isfinite(log_alpha) ? expf(fminf(log_alpha, 0.0f)) : 0.0f;
}

// ---------------------------------------------------------------------------
// Dual averaging (Hoffman and Gelman 2014, Section 3.2.1 / Algorithm 5), one
// step size per posterior, updated once per burn-in transition from the mean
// over chains of min(1, alpha).  Lives in device memory so that a captured
// sampling loop never returns to the host.
// ---------------------------------------------------------------------------
struct DAState {
  double log_eps;       // step size of the next transition (log)
  double log_eps_bar;   // running average, frozen step size after adaptation
  double h_bar;         // running mean of (delta - alpha)
  double mu;            // shrinkage point log(10 eps0)
  double delta;         // target acceptance
  double last_stat;     // statistic of the last transition (diagnostic)
  long long m;          // adaptation steps taken
  long long num_adapt;  // transitions with t < num_adapt adapt
  float eps;            // float32 copy of exp(log_eps) read by the kernels
  int adapt;            // 0: fixed step size
  unsigned int arrive;  // blocks of the current transition that finished
  unsigned int pad;
};

constexpr double kDAGamma = 0.05;
constexpr double kDAT0 = 10.0;
constexpr double kDAKappa = 0.75;

// The coefficients of adaptation step m depend on m alone, so a kernel can
// form them before the acceptance statistic exists: w = 1 / (m + t0),
// sqrt(m) / gamma and eta = m^-kappa (kappa = 3/4: m^-1/2 m^-1/4).  Float64
// is slow on this part, so the kernels keep these off the critical path.
struct DACoef {
  double w, sq, eta;
  int active;      // 0: transition t does not adapt
};
static_assert(kDAKappa == 0.75, "eta below is m^-3/4");

__device__ __forceinline__ DACoef da_prepare(const DAState* s, long long t) {
  DACoef c{0.0, 0.0, 0.0, 0};
  if (!s->adapt || t >= s->num_adapt) return c;
  const double m = static_cast<double>(s->m + 1);
  const double r = sqrt(m);
  c.w = 1.0 / (m + kDAT0);
  c.sq = r / kDAGamma;
  c.eta = 1.0 / (r * sqrt(r));
  c.active = 1;
  return c;
}

// Apply one adaptation step with statistic `alpha` after transition t.
__device__ __forceinline__ void da_apply(DAState* s, const DACoef& c, double alpha, long long t) {
  s->last_stat = alpha;
  if (!c.active) return;
  s->m += 1;
  // explicit roundings: no multiply-add contraction, so every kernel that
  // inlines this takes the same steps (and float64 evaluates as written)
  s->h_bar = __dadd_rn(__dmul_rn(1.0 - c.w, s->h_bar), __dmul_rn(c.w, __dsub_rn(s->delta, alpha)));
  s->log_eps = __dsub_rn(s->mu, __dmul_rn(c.sq, s->h_bar));
  s->log_eps_bar = __dadd_rn(__dmul_rn(c.eta, s->log_eps), __dmul_rn(1.0 - c.eta, s->log_eps_bar));
  // after the last adaptation step the step size freezes at eps_bar; the
  // kernels use the step size as float32, formed by a float32 exp of the
  // rounded logarithm (within 3e-7 of float64 exp, which is slow on this
  // part and sits on the critical path of every adapting transition)
  const double next = (t + 1 >= s->num_adapt) ? s->log_eps_bar : s->log_eps;
  s->eps = expf(static_cast<float>(next));
}

__device__ __forceinline__ void da_update(DAState* s, double alpha, long long t) {
  da_apply(s, da_prepare(s, t), alpha, t);
}

// Deterministic reduction of per-tile partial sums followed by the
// dual-averaging update: every tile (CTA) of a posterior stores its partial,
// the last tile to arrive sums all partials in tile order (so the result does
// not depend on arrival order), updates the state and re-arms the counter.
// `tile` / `ntiles` index the CTAs of this posterior (the whole grid when one
// launch serves one posterior).  Returns, in every thread, whether this block
// applied the update.
__device__ __forceinline__ bool tile_partial_then_da(DAState* s, double* partials, double block_sum,
                                                     int num_chains, long long t, int tile,
                                                     int ntiles) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[tile] = block_sum;
    __threadfence();
    const unsigned int prev = atomicAdd(&s->arrive, 1u);
    last = (prev == static_cast<unsigned int>(ntiles) - 1u);
  }
  __syncthreads();
  const bool mine = last;
  if (!mine) return false;
  __threadfence();
  double acc = 0.0;
  if (threadIdx.x < 32) {
    for (int b = threadIdx.x; b < ntiles; b += 32) acc += static_cast<volatile double*>(partials)[b];
    acc = warp_sum_d(acc);
    if (threadIdx.x == 0) {
      da_update(s, acc / static_cast<double>(num_chains), t);
      s->arrive = 0u;
      __threadfence();
    }
  }
  return true;
}

__device__ __forceinline__ void block_partial_then_da(DAState* s, double* partials, double block_sum,
                                                      int num_chains, long long t) {
  tile_partial_then_da(s, partials, block_sum, num_chains, t, static_cast<int>(blockIdx.x),
                       static_cast<int>(gridDim.x));
}

// Sum of one acceptance probability per warp of this block (warps with no
// chain pass has_chain = false), in warp order, then the deterministic grid
// reduction and dual-averaging update.
template <int kWarps>
__device__ __forceinline__ bool accept_tile_finish(DAState* da, double* partials, float prob,
                                                   bool has_chain, int num_chains, long long t,
                                                   int tile, int ntiles) {
  __shared__ float warp_prob[kWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) warp_prob[w] = has_chain ? prob : 0.f;
  __syncthreads();
  double sum = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kWarps; ++i) sum += static_cast<double>(warp_prob[i]);
  return tile_partial_then_da(da, partials, sum, num_chains, t, tile, ntiles);
}

template <int kWarps>
__device__ __forceinline__ void accept_block_finish(DAState* da, double* partials, float prob,
                                                    bool has_chain, int num_chains, long long t) {
  accept_tile_finish<kWarps>(da, partials, prob, has_chain, num_chains, t,
                             static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
}

// Welford's running mean and sum of squared deviations (Welford 1962) of the
// kept draws 0..k of one element, and, with bsize > 0, the same recursion
// over the means of consecutive batches of bsize draws (bsum accumulates
// the current batch; at its last draw the batch mean enters bmean / bm2).
// The per-draw constants are formed once per kept transition.
struct WelfordCoef {
  float inv, inv_b, inv_j;
  int64_t pos, batch;
  bool closes;
};

__device__ __forceinline__ WelfordCoef welford_coef(int64_t k, int64_t bsize) {
  WelfordCoef q;
  q.inv = 1.0f / static_cast<float>(k + 1);
  q.pos = bsize > 0 ? k % bsize : 0;
  q.batch = bsize > 0 ? k / bsize : 0;
  q.closes = bsize > 0 && q.pos == bsize - 1;
  q.inv_b = bsize > 0 ? 1.0f / static_cast<float>(bsize) : 0.f;
  q.inv_j = 1.0f / static_cast<float>(q.batch + 1);
  return q;
}

template <typename W>
__device__ __forceinline__ void welford_update(const W& w, const WelfordCoef& q, int64_t k, int64_t i,
                                               float v) {
  if (k == 0) {
    w.mean[i] = v;
    w.m2[i] = 0.f;
  } else {
    const float m0 = w.mean[i];
    const float delta = v - m0;
    const float m1 = fmaf(delta, q.inv, m0);
    w.mean[i] = m1;
    w.m2[i] = fmaf(delta, v - m1, w.m2[i]);
  }
  if (w.bsize > 0) {
    const float sum = q.pos == 0 ? v : w.bsum[i] + v;
    w.bsum[i] = sum;
    if (q.closes) {
      const float bm = sum * q.inv_b;
      if (q.batch == 0) {
        w.bmean[i] = bm;
        w.bm2[i] = 0.f;
      } else {
        const float b0 = w.bmean[i];
        const float delta = bm - b0;
        const float b1 = fmaf(delta, q.inv_j, b0);
        w.bmean[i] = b1;
        w.bm2[i] = fmaf(delta, bm - b1, w.bm2[i]);
      }
    }
  }
}

// welford_update for N elements with every load issued before any store, so
// that the N read-modify-writes overlap instead of each waiting for its
// predecessor's stores (the compiler cannot tell that the elements' arrays
// do not alias).  Element j is skipped unless bit j of `valid` is set.
template <int N, typename W>
__device__ __forceinline__ void welford_update_n(const W& w, const WelfordCoef& q, int64_t k,
                                                 const int64_t (&idx)[N], const float (&v)[N],
                                                 uint32_t valid) {
  float m0[N], s0[N], b0[N], bm0[N], bs0[N];
  const bool batches = w.bsize > 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    m0[j] = s0[j] = b0[j] = bm0[j] = bs0[j] = 0.f;
    if (!((valid >> j) & 1u)) continue;
    if (k > 0) {
      m0[j] = w.mean[idx[j]];
      s0[j] = w.m2[idx[j]];
    }
    if (batches && q.pos != 0) b0[j] = w.bsum[idx[j]];
    if (batches && q.closes && q.batch > 0) {
      bm0[j] = w.bmean[idx[j]];
      bs0[j] = w.bm2[idx[j]];
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (!((valid >> j) & 1u)) continue;
    const float x = v[j];
    if (k == 0) {
      w.mean[idx[j]] = x;
      w.m2[idx[j]] = 0.f;
    } else {
      const float delta = x - m0[j];
      const float m1 = fmaf(delta, q.inv, m0[j]);
      w.mean[idx[j]] = m1;
      w.m2[idx[j]] = fmaf(delta, x - m1, s0[j]);
    }
    if (batches) {
      const float sum = q.pos == 0 ? x : b0[j] + x;
      w.bsum[idx[j]] = sum;
      if (q.closes) {
        const float bm = sum * q.inv_b;
        if (q.batch == 0) {
          w.bmean[idx[j]] = bm;
          w.bm2[idx[j]] = 0.f;
        } else {
          const float delta = bm - bm0[j];
          const float b1 = fmaf(delta, q.inv_j, bm0[j]);
          w.bmean[idx[j]] = b1;
          w.bm2[idx[j]] = fmaf(delta, bm - b1, bs0[j]);
        }
      }
    }
  }
}

// Logistic regression (the tensor-core products' epilogues).  y - sigmoid(z)
// for the gradient with the fast exponential and divide (a few ulp; the
// gradient tolerance is orders of magnitude looser):
__device__ __forceinline__ float residual_f(float y, float z) {
  const float e = __expf(-fabsf(z));
  const float inv = __fdividef(1.f, 1.f + e);
  return y - (z >= 0.f ? inv : e * inv);
}

// y z - softplus(z) for log p, correctly rounded building blocks (the
// accept test compares sums over all rows)
__device__ __forceinline__ float loglik_f(float y, float z) {
  return y * z - (fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))));
}

// Split x into its tf32 head (10 explicit mantissa bits) and the exact float32
// remainder: x = hi + lo exactly.  Used by the 3xTF32 products.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

}  // namespace hmc
