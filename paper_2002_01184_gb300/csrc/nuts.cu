// The No-U-Turn Sampler with the recursion unrolled (Section 2.3), for the
// targets whose gradient is elementwise plus row reductions (standard
// normal, funnel).  One warp per chain, one launch per transition; chains
// build their trees independently, so a warp's lanes never diverge and
// different chains' tree sizes cost nothing to each other.
//
// The transition is Hoffman and Gelman's efficient NUTS (slice variable u)
// as a loop: doubling j grows a subtree of 2^j leapfrog steps (step v_j eps)
// from the trajectory's end on side v_j; at leaf k every span of 2^i leaves
// that closes is checked for a U-turn against its first leaf, which is the
// only state kept per level -- O(max_depth) states, not the 2^depth
// trajectory.  The chain's working (x, p, g) lives in registers (lane owns
// dims 4 (lane + 32 b) .. + 3); the two trajectory ends, the two candidates
// and the span starts live in a per-chain scratch of 30 slots of D floats.
//
// Random choices: directions from word 0 of counter (0, chain, t, 3), the
// subtree's choice at leaf k of doubling j from counter (k, chain, t, 4 + j),
// the top-level choice at doubling j from counter (j, chain, t, 14); a choice
// of probability a / b is taken iff (2 w + 1) b < a 2^33 (exact integers).
#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"

namespace hmc {

namespace {

constexpr int kWarps = 8;
constexpr uint32_t kTagDirection = 3u, kTagSubtree = 4u, kTagTop = 14u;
constexpr float kDeltaMax = 1000.f;
// slots: 0-2 left end x, p, g; 3-5 right end; 6-7 candidate x, g;
// 8-9 subtree candidate x, g; 10 + 2 (i - 1), + 1: first leaf x, p of level i
constexpr int kSlotLeft = 0, kSlotRight = 3, kSlotCand = 6, kSlotSub = 8, kSlotSpan = 10;

__device__ __forceinline__ uint32_t word0(uint64_t seed, uint32_t w, uint32_t chain, uint32_t t,
                                          uint32_t tag) {
  return philox(make_uint4(w, chain, t, tag), static_cast<uint32_t>(seed),
                static_cast<uint32_t>(seed >> 32)).x;
}

// probability a / b, b > 0: (2 w + 1) b < a 2^33
__device__ __forceinline__ bool take(uint32_t w, uint32_t a, uint32_t b) {
  return (2ull * w + 1ull) * b < (static_cast<unsigned long long>(a) << 33);
}

struct NutsArgs {
  StepArgs s;
  float* scratch;                  // [C][kNutsSlots][Dp]
  int Dp;                          // D rounded up to 4
  int max_depth;
  unsigned long long* leaves;      // total leapfrog steps (gradient evaluations)
};

template <int TARGET, int NB>
__global__ void __launch_bounds__(32 * kWarps) k_nuts(NutsArgs na) {
  const StepArgs& a = na.s;
  const int c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) {
    const int D = a.D;
    const int64_t row = static_cast<int64_t>(c) * D;
    const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
    const float eps = a.da->eps;
    float* base = na.scratch + static_cast<int64_t>(c) * kNutsSlots * na.Dp;
    float x[NB][4], p[NB][4], g[NB][4];
    auto slot4 = [&](int s, int b) {
      return reinterpret_cast<float4*>(base + static_cast<int64_t>(s) * na.Dp) + (lane + 32 * b);
    };
    auto in_slot = [&](int b) { return 4 * (lane + 32 * b) < na.Dp; };
    auto store = [&](int s, const float (&v)[NB][4]) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (in_slot(b)) *slot4(s, b) = make_float4(v[b][0], v[b][1], v[b][2], v[b][3]);
    };
    auto load = [&](int s, float (&v)[NB][4]) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in_slot(b)) q = *slot4(s, b);
        v[b][0] = q.x; v[b][1] = q.y; v[b][2] = q.z; v[b][3] = q.w;
      }
    };
    auto dot = [&](const float (&u)[NB][4], const float (&w)[NB][4]) {
      float acc = 0.f;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc = fmaf(u[b][i], w[b][i], acc);
      return warp_sum(acc);
    };
    // log p and gradient at x (dims past D stay zero)
    const float half_n = 0.5f * static_cast<float>(D - 1);
    auto target = [&]() {
      float q = 0.f;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bool is_v = TARGET == HMC_T_FUNNEL && b == 0 && i == 0 && lane == 0;
          q = is_v ? q : fmaf(x[b][i], x[b][i], q);
        }
      if (TARGET == HMC_T_STD_NORMAL) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) g[b][i] = -x[b][i];
        return -0.5f * warp_sum(q);
      } else {
        const float v = __shfl_sync(0xffffffffu, x[0][0], 0);
        q = warp_sum(q);
        const float ev = expf(-v);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) g[b][i] = -ev * x[b][i];
        if (lane == 0) g[0][0] = -v / 9.f - half_n + 0.5f * ev * q;
        return -v * v / 18.f - half_n * v - 0.5f * ev * q;
      }
    };

    // start: x0, g0, p0 ~ N(0, I), H0, log U
    float lp = a.lp[c];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = lane + 32 * b;
      const float4 z = momentum4(a.seed, static_cast<uint32_t>(j), chain, a.t);
      const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * j + i;
        const bool in = d < D;
        x[b][i] = in ? a.x[row + d] : 0.f;
        g[b][i] = in ? a.g[row + d] : 0.f;
        p[b][i] = in ? zz[i] : 0.f;
      }
    }
    const float H0 = -lp + 0.5f * dot(p, p);
    const float logU = accept_log_uniform(a.seed, chain, a.t);
    store(kSlotLeft, x); store(kSlotLeft + 1, p); store(kSlotLeft + 2, g);
    store(kSlotRight, x); store(kSlotRight + 1, p); store(kSlotRight + 2, g);
    store(kSlotCand, x); store(kSlotCand + 1, g);
    float lp_end[2] = {lp, lp};     // [0]: left, [1]: right
    float lpm = lp;
    uint32_t n = 1;
    int moved = 0;
    float a_sum = 0.f;
    uint32_t n_a = 0;
    const uint32_t dirs = word0(a.seed, 0u, chain, a.t, kTagDirection);
    for (int jd = 0; jd < na.max_depth; ++jd) {
      const int v = ((dirs >> jd) & 1u) ? 1 : -1;
      const float ev = static_cast<float>(v) * eps;
      const int side = v > 0 ? kSlotRight : kSlotLeft;
      load(side, x); load(side + 1, p); load(side + 2, g);
      lp = lp_end[v > 0 ? 1 : 0];
      uint32_t n_sub = 0;
      bool ok_sub = true;
      float lps = 0.f;
      const int leaves = 1 << jd;
      for (int k = 0; k < leaves; ++k) {
        // one leapfrog step of step v eps
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            p[b][i] = fmaf(0.5f * ev, g[b][i], p[b][i]);
            x[b][i] = fmaf(ev, p[b][i], x[b][i]);
          }
        lp = target();
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) p[b][i] = fmaf(0.5f * ev, g[b][i], p[b][i]);
        const float H = -lp + 0.5f * dot(p, p);
        const bool finite = isfinite(H);
        if (!finite || H - H0 >= kDeltaMax - logU) ok_sub = false;     // divergence
        a_sum += finite ? accept_prob(H0 - H) : 0.f;
        ++n_a;
        if (finite && logU <= H0 - H) {
          ++n_sub;
          if (take(word0(a.seed, static_cast<uint32_t>(k), chain, a.t, kTagSubtree + jd), 1u, n_sub)) {
            store(kSlotSub, x);
            store(kSlotSub + 1, g);
            lps = lp;
          }
        }
        // spans of 2^i leaves opening / closing at leaf k
        for (int i = 1; i <= jd; ++i) {
          const int span = 1 << i;
          const int s = kSlotSpan + 2 * (i - 1);
          if (k % span == 0) {
            store(s, x);
            store(s + 1, p);
          }
          if ((k + 1) % span == 0) {
            float xf[NB][4], pf[NB][4], dx[NB][4];
            load(s, xf);
            load(s + 1, pf);
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
              for (int q = 0; q < 4; ++q) dx[b][q] = static_cast<float>(v) * (x[b][q] - xf[b][q]);
            if (dot(dx, pf) < 0.f || dot(dx, p) < 0.f) ok_sub = false;
          }
        }
        if (!ok_sub) break;
      }
      store(side, x); store(side + 1, p); store(side + 2, g);
      lp_end[v > 0 ? 1 : 0] = lp;
      if (!ok_sub) break;
      if (n_sub > 0 && take(word0(a.seed, static_cast<uint32_t>(jd), chain, a.t, kTagTop), n_sub, n)) {
        float t1[NB][4], t2[NB][4];
        load(kSlotSub, t1);
        load(kSlotSub + 1, t2);
        store(kSlotCand, t1);
        store(kSlotCand + 1, t2);
        lpm = lps;
        moved = 1;
      }
      n += n_sub;
      // the whole trajectory's ends
      float xl[NB][4], pl[NB][4], xr[NB][4], pr[NB][4];
      load(kSlotLeft, xl); load(kSlotLeft + 1, pl);
      load(kSlotRight, xr); load(kSlotRight + 1, pr);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) xr[b][q] -= xl[b][q];
      if (dot(xr, pl) < 0.f || dot(xr, pr) < 0.f) break;
    }
    // the new state
    load(kSlotCand, x);
    load(kSlotCand + 1, g);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = lane + 32 * b;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * j + i;
        if (d < D) {
          a.x[row + d] = x[b][i];
          a.g[row + d] = g[b][i];
          if (a.sample_out) a.sample_out[row + d] = x[b][i];
        }
      }
    }
    prob = a_sum / static_cast<float>(n_a);
    if (lane == 0) {
      a.lp[c] = lpm;
      a.is_accepted[c] = static_cast<uint8_t>(moved);
      a.log_accept[c] = logf(prob);
      if (a.trace_acc) a.trace_acc[c] = static_cast<uint8_t>(moved);
      if (c == 0 && a.trace_eps) a.trace_eps[0] = eps;
      atomicAdd(na.leaves, static_cast<unsigned long long>(n_a));
    }
  }
  accept_tile_finish<kWarps>(a.da, a.partials, prob, has_chain, a.C, a.t_full,
                             static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
}

template <int TARGET>
cudaError_t launch_t(const NutsArgs& na, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>((na.s.C + kWarps - 1) / kWarps);
  const int nb = (na.s.D + 127) / 128;
  if (nb <= 1) k_nuts<TARGET, 1><<<grid, 32 * kWarps, 0, s>>>(na);
  else if (nb == 2) k_nuts<TARGET, 2><<<grid, 32 * kWarps, 0, s>>>(na);
  else k_nuts<TARGET, 4><<<grid, 32 * kWarps, 0, s>>>(na);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool nuts_supported(const hmc_target& t) {
  return (t.id == HMC_T_STD_NORMAL || t.id == HMC_T_FUNNEL) && t.dim <= kNutsMaxDim;
}

size_t nuts_scratch_floats(const hmc_target& t, int64_t C) {
  return static_cast<size_t>(C) * kNutsSlots * ((t.dim + 3) / 4 * 4);
}

cudaError_t launch_nuts_transition(const hmc_target& t, const StepArgs& a, float* scratch,
                                   int max_depth, unsigned long long* leaves, cudaStream_t s,
                                   KernelTimer* timer) {
  NutsArgs na{a, scratch, (t.dim + 3) / 4 * 4, max_depth, leaves};
  if (timer) timer->begin(s);
  cudaError_t e = t.id == HMC_T_FUNNEL ? launch_t<HMC_T_FUNNEL>(na, s) : launch_t<HMC_T_STD_NORMAL>(na, s);
  if (timer) timer->end(s);
  return e;
}

}  // namespace hmc
