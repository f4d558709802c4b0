// Fused HMC transition for targets whose gradient is elementwise plus row
// reductions (standard normal, funnel), as a tile function: one CTA of 256
// threads advances 8 chains (one warp each) through momentum draw, L leapfrog
// steps and the Metropolis-Hastings select (Section 2.1), with each chain's
// x, p and g in its warp's registers.  `tile` indexes the CTA among the
// `ntiles` CTAs of its posterior (for the shared dual-averaging reduction).
#pragma once
#include "hmc_device.cuh"
#include "hmc_internal.h"

namespace hmc {

// Lane `lane` of the chain's warp owns Philox blocks j = lane + 32 b
// (b < NB), i.e. state dims 4 j .. 4 j + 3.
// With reduce = false the tile skips its share of the dual-averaging
// reduction (a transition whose statistic nobody needs); returns whether this
// tile applied the update.
template <int TARGET, int NB>
__device__ __forceinline__ bool elementwise_tile(const StepArgs& a, int tile, int ntiles, bool reduce = true) {
  constexpr int kWarpsPerBlock = 8;
  const int c = tile * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) {
    const int D = a.D;
    const int64_t row = static_cast<int64_t>(c) * D;
    const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
    const float eps = a.da->eps;
    float x0[NB][4], x[NB][4], p[NB][4], g[NB][4];
    float kin0 = 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = lane + 32 * b;
      const float4 z = momentum4(a.seed, static_cast<uint32_t>(j), chain, a.t);
      const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * j + i;
        const bool in = d < D;
        x0[b][i] = in ? a.x[row + d] : 0.f;
        x[b][i] = x0[b][i];
        g[b][i] = in ? a.g[row + d] : 0.f;
        p[b][i] = in ? zz[i] : 0.f;
        kin0 = fmaf(p[b][i], p[b][i], kin0);
      }
    }
    kin0 = 0.5f * warp_sum(kin0);
    const float lp0 = a.lp[c];
    float lp1 = 0.f;
    const float half_n = 0.5f * static_cast<float>(D - 1);
    for (int l = 0; l < a.L; ++l) {
      float q = 0.f;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          p[b][i] = fmaf(0.5f * eps, g[b][i], p[b][i]);
          x[b][i] = fmaf(eps, p[b][i], x[b][i]);
          // the funnel's reduction runs over x_1.. only (dim 0 is v)
          const bool is_v = TARGET == HMC_T_FUNNEL && b == 0 && i == 0 && lane == 0;
          q = is_v ? q : fmaf(x[b][i], x[b][i], q);
        }
      if (TARGET == HMC_T_STD_NORMAL) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) g[b][i] = -x[b][i];
        if (l == a.L - 1) lp1 = -0.5f * warp_sum(q);
      } else {  // funnel: v is dim 0 (lane 0, block 0, word 0)
        const float v = __shfl_sync(0xffffffffu, x[0][0], 0);
        q = warp_sum(q);
        const float ev = expf(-v);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) g[b][i] = -ev * x[b][i];
        if (lane == 0) g[0][0] = -v / 9.f - half_n + 0.5f * ev * q;
        if (l == a.L - 1) lp1 = -v * v / 18.f - half_n * v - 0.5f * ev * q;
      }
      if (a.K > 1) {      // replica exchange: this row targets p^beta
        const float beta = a.betas[c % a.K];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) g[b][i] *= beta;
        if (l == a.L - 1) lp1 *= beta;
      }
      // dims past D keep x = p = g = 0 throughout (g = -x and -e^-v x vanish)
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          p[b][i] = fmaf(0.5f * eps, g[b][i], p[b][i]);
        }
    }
    float kin1 = 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int i = 0; i < 4; ++i) kin1 = fmaf(p[b][i], p[b][i], kin1);
    kin1 = 0.5f * warp_sum(kin1);
    const float h0 = -lp0 + kin0, h1 = -lp1 + kin1;
    float la = h0 - h1;
    if (!isfinite(la)) la = -INFINITY;
    int acc = 0;
    if (lane == 0) acc = accept_log_uniform(a.seed, chain, a.t) < la;
    acc = __shfl_sync(0xffffffffu, acc, 0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = lane + 32 * b;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * j + i;
        if (d < D) {
          if (acc) {
            a.x[row + d] = x[b][i];
            a.g[row + d] = g[b][i];
          }
          if (a.sample_out) a.sample_out[row + d] = acc ? x[b][i] : x0[b][i];
        }
      }
    }
    if (lane == 0) {
      if (acc) a.lp[c] = lp1;
      a.is_accepted[c] = static_cast<uint8_t>(acc);
      a.log_accept[c] = la;
      if (a.trace_acc) a.trace_acc[c] = static_cast<uint8_t>(acc);
      if (c == 0 && a.trace_eps) a.trace_eps[0] = eps;
    }
    prob = accept_prob(la);
  }
  if (!reduce) return false;
  return accept_tile_finish<kWarpsPerBlock>(a.da, a.partials, prob, has_chain, a.C, a.t_full, tile, ntiles);
}


}  // namespace hmc
