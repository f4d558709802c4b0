// Fused HMC transition for Bayesian logistic regression as a tile function
// (Section 2.1's transition with the batched target of a "list of vectors"):
// one CTA owns kLrTC chains for the whole transition -- momentum draw, L
// leapfrog steps, Metropolis-Hastings select -- with positions, momenta and
// gradients in shared memory.  Each gradient streams the data X in tiles of
// kLrRT rows through shared memory; every tile serves all of the CTA's chains:
//   z[r][c] = <X_r, theta_c>           (two threads per (row, chain) pair)
//   res[r][c] = y_r - sigmoid(z)        lp partial += y_r z - softplus(z)
//   g[c][:] += sum_r res[r][c] X_r      (warp c, lanes along the dims)
// then g -= theta (the N(0, I) prior) and lp -= |theta|^2 / 2.  Float32
// SIMT arithmetic, dim <= kLrMaxDim.
#pragma once
#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"

namespace hmc {
namespace lr {

constexpr int kLrTC = 8;          // chains per CTA (one warp each for elementwise work)
constexpr int kLrRT = 16;         // data rows per tile
constexpr int kLrThreads = 256;
constexpr int kLrMaxDim = 512;

struct LrArgs {
  StepArgs s;
  const float* X;
  const float* y;
  int N;
};

// gradient residual with the fast exponential and divide (a few ulp)
__device__ __forceinline__ float sigmoid_stable(float z) {
  const float e = __expf(-fabsf(z));
  const float inv = __fdividef(1.f, 1.f + e);
  return z >= 0.f ? inv : e * inv;
}

__device__ __forceinline__ float softplus_stable(float z) {
  return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
}

// Shared-memory layout (floats), row stride ld = D + 1 (odd: the eight chain
// rows read at one column fall in distinct banks).
struct Smem {
  float* th;    // [kLrTC][ld] positions
  float* pm;    // [kLrTC][ld] momenta
  float* gr;    // [kLrTC][ld] gradient
  float* Xs;    // [kLrRT][ld] data tile
  float* ys;    // [kLrRT]
  float* res;   // [kLrRT][kLrTC]
  float* lpb;   // [kLrRT * kLrTC] per-(row, chain) log-lik partials
  float* red;   // [kLrTC] per-chain scalars
};

__device__ __forceinline__ Smem carve(float* base, int ld) {
  Smem s;
  s.th = base;
  s.pm = s.th + kLrTC * ld;
  s.gr = s.pm + kLrTC * ld;
  s.Xs = s.gr + kLrTC * ld;
  s.ys = s.Xs + kLrRT * ld;
  s.res = s.ys + kLrRT;
  s.lpb = s.res + kLrRT * kLrTC;
  s.red = s.lpb + kLrRT * kLrTC;
  return s;
}

// gr[c] = grad log p(th_c); with need_lp also log p(th_c) in red[c] (all
// threads call; log p is needed at the end of a trajectory only)
__device__ __noinline__ static void gradient(const LrArgs& a, const Smem& s, int ld, int nvalid,
                                             bool need_lp) {
  const int D = a.s.D, N = a.N;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  for (int d = lane; d < D; d += 32) s.gr[w * ld + d] = 0.f;
  const int pair = t >> 1, half = t & 1;
  const int pr = pair >> 3, pc = pair & 7;
  float lp_acc = 0.f;
  for (int r0 = 0; r0 < N; r0 += kLrRT) {
    const int rows = min(kLrRT, N - r0);
    const float* src = a.X + static_cast<int64_t>(r0) * D;
    for (int e = t; e < kLrRT * D; e += kLrThreads) {
      const int r = e / D, d = e - r * D;
      s.Xs[r * ld + d] = r < rows ? src[e] : 0.f;
    }
    if (t < kLrRT) s.ys[t] = t < rows ? a.y[r0 + t] : 0.f;
    __syncthreads();
    float z = 0.f;
    for (int d = half; d < D; d += 2) z = fmaf(s.Xs[pr * ld + d], s.th[pc * ld + d], z);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    if (half == 0) {
      float r = 0.f;
      if (pr < rows && pc < nvalid) {
        const float yv = s.ys[pr];
        r = yv - sigmoid_stable(z);
        if (need_lp) lp_acc += yv * z - softplus_stable(z);
      }
      s.res[pr * kLrTC + pc] = r;
    }
    __syncthreads();
    for (int d = lane; d < D; d += 32) {
      float acc = 0.f;
#pragma unroll
      for (int r = 0; r < kLrRT; ++r) acc = fmaf(s.res[r * kLrTC + w], s.Xs[r * ld + d], acc);
      s.gr[w * ld + d] += acc;
    }
    __syncthreads();
  }
  if (half == 0) s.lpb[pr * kLrTC + pc] = lp_acc;
  __syncthreads();
  // prior: g -= theta, lp -= |theta|^2 / 2; per-chain sums in row order
  float sq = 0.f;
  for (int d = lane; d < D; d += 32) {
    const float th = s.th[w * ld + d];
    s.gr[w * ld + d] -= th;
    sq = fmaf(th, th, sq);
  }
  sq = warp_sum(sq);
  if (lane == 0) {
    float lp = 0.f;
    for (int r = 0; r < kLrRT; ++r) lp += s.lpb[r * kLrTC + w];
    s.red[w] = lp - 0.5f * sq;
  }
  __syncthreads();
}

// One CTA of kLrThreads threads: chains tile * kLrTC .. + kLrTC of the posterior.
// With reduce = false the tile skips its share of the dual-averaging
// reduction; returns whether this tile applied the update.
__device__ __forceinline__ bool logreg_tile(const LrArgs& a, int tile, int ntiles, bool reduce = true) {
  extern __shared__ float smem_f[];
  const StepArgs& A = a.s;
  const int D = A.D, C = A.C;
  const int ld = D + 1;
  const Smem s = carve(smem_f, ld);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int c0 = tile * kLrTC;
  const int nvalid = min(kLrTC, C - c0);
  const int chain = c0 + w;
  const bool has_chain = w < nvalid;
  const int64_t row = static_cast<int64_t>(chain) * D;
  const float eps = A.da->eps;
  const uint32_t gchain = static_cast<uint32_t>(chain) + A.chain_offset;

  // begin: p0 ~ N(0, I), K0, half kick with the cached gradient, first drift
  float kin0 = 0.f;
  for (int d = lane; d < D; d += 32) {
    float x = 0.f, g = 0.f, z = 0.f;
    if (has_chain) {
      x = A.x[row + d];
      g = A.g[row + d];
      z = momentum1(A.seed, static_cast<uint32_t>(d), gchain, A.t);
    }
    kin0 = fmaf(z, z, kin0);
    const float p = fmaf(0.5f * eps, g, z);
    s.pm[w * ld + d] = p;
    s.th[w * ld + d] = fmaf(eps, p, x);
  }
  kin0 = 0.5f * warp_sum(kin0);
  __syncthreads();
  for (int l = 1; l <= A.L; ++l) {
    gradient(a, s, ld, nvalid, l == A.L);
    const float kick = l < A.L ? eps : 0.5f * eps;
    for (int d = lane; d < D; d += 32) {
      const float p = fmaf(kick, s.gr[w * ld + d], s.pm[w * ld + d]);
      s.pm[w * ld + d] = p;
      if (l < A.L) s.th[w * ld + d] = fmaf(eps, p, s.th[w * ld + d]);
    }
    __syncthreads();
  }
  float prob = 0.f;
  if (has_chain) {
    float kin1 = 0.f;
    for (int d = lane; d < D; d += 32) kin1 = fmaf(s.pm[w * ld + d], s.pm[w * ld + d], kin1);
    kin1 = 0.5f * warp_sum(kin1);
    const float lp0 = A.lp[chain];
    const float lp1 = s.red[w];
    float la = (-lp0 + kin0) - (-lp1 + kin1);
    if (!isfinite(la)) la = -INFINITY;
    int acc = 0;
    if (lane == 0) acc = accept_log_uniform(A.seed, gchain, A.t) < la;
    acc = __shfl_sync(0xffffffffu, acc, 0);
    for (int d = lane; d < D; d += 32) {
      if (acc) {
        A.x[row + d] = s.th[w * ld + d];
        A.g[row + d] = s.gr[w * ld + d];
      }
      if (A.sample_out) A.sample_out[row + d] = A.x[row + d];
    }
    if (lane == 0) {
      if (acc) A.lp[chain] = lp1;
      A.is_accepted[chain] = static_cast<uint8_t>(acc);
      A.log_accept[chain] = la;
      if (A.trace_acc) A.trace_acc[chain] = static_cast<uint8_t>(acc);
      if (chain == 0 && A.trace_eps) A.trace_eps[0] = eps;
    }
    prob = accept_prob(la);
  }
  if (!reduce) return false;
  return accept_tile_finish<kLrThreads / 32>(A.da, A.partials, prob, has_chain, C, A.t_full, tile, ntiles);
}

inline size_t logreg_smem_bytes(int D) {
  const int ld = D + 1;
  return sizeof(float) * (3 * kLrTC * ld + kLrRT * ld + kLrRT + 2 * kLrRT * kLrTC + kLrTC);
}


}  // namespace lr
}  // namespace hmc
