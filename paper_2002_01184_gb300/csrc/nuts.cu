// The No-U-Turn Sampler with the recursion unrolled (Section 2.3), for the
// targets whose gradient is elementwise plus row reductions (standard
// normal, funnel).  One warp per chain; chains build their trees
// independently, so a warp's lanes never diverge and different chains' tree
// sizes cost nothing to each other.  A launch runs one transition, or -- where
// the step size is fixed (no adaptation in the range) -- a run of
// transitions, so that each chain's tree sizes average out over the run
// instead of every transition waiting for the deepest tree of all chains.
//
// The transition is Hoffman and Gelman's efficient NUTS (slice variable u)
// as a loop: doubling j grows a subtree of 2^j leapfrog steps (step v_j eps)
// from the trajectory's end on side v_j; at leaf k every span of 2^i leaves
// that closes is checked for a U-turn against its first leaf, which is the
// only state kept per level -- O(max_depth) states, not the 2^depth
// trajectory.  The chain's working (x, p, g) lives in registers (lane owns
// dims 4 (lane + 32 b) .. + 3); the span starts live in shared memory where
// the occupancy allows (else in the per-chain scratch), the two trajectory
// ends and the two candidates in a per-chain scratch of kNutsSlots slots of
// D floats.
//
// The random streams and the choice rule are those of nuts_common.cuh.
#include <cmath>

#include "nuts_common.cuh"

namespace hmc {

namespace {

constexpr int kWarps = 4;

struct NutsArgs {
  StepArgs s;                      // transition s.t_full is the launch's first
  float* scratch;                  // [C][kNutsSlots][Dp]
  int Dp;                          // D rounded up to 4
  int max_depth;
  unsigned long long* leaves;      // [0] leapfrog steps (gradient evaluations), [1] critical
                                   // path (the launches' longest chains), [2] this launch's longest
  int T;                           // transitions in this launch (T > 1: none adapts)
  long long keep_from;             // transition whose new state is kept sample 0
  float* samples;                  // [K][C][D] kept states, or null
  float* trace_eps;                // [K] step size per kept transition, or null
  uint8_t* trace_acc;              // [K][C] moved flags, or null
};

// shared-memory span starts: 2 (max_depth - 1) rows of Dp floats per warp
size_t span_smem_bytes(int Dp, int max_depth) {
  return static_cast<size_t>(kWarps) * 2 * (max_depth > 1 ? max_depth - 1 : 0) * Dp * sizeof(float);
}

// residency: 7 blocks (28 warps, 4256 chains on 152 SMs) per SM at NB = 1, 4
// at NB = 2, 4 (registers)
template <int TARGET, int NB, bool SMEM>
__global__ void __launch_bounds__(32 * kWarps, NB == 1 ? 7 : 4) k_nuts(NutsArgs na) {
  extern __shared__ float4 span_smem[];
  const StepArgs& a = na.s;
  const int warp = threadIdx.x >> 5;
  const int c = blockIdx.x * kWarps + warp;
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) {
    const int D = a.D;
    const int64_t row = static_cast<int64_t>(c) * D;
    const int64_t CD = static_cast<int64_t>(a.C) * D;
    const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
    const float eps = a.da->eps;
    float* base = na.scratch + static_cast<int64_t>(c) * kNutsSlots * na.Dp;
    float4* spans = span_smem + static_cast<int64_t>(warp) * 2 * (na.max_depth - 1) * (na.Dp / 4);
    float x[NB][4], p[NB][4], g[NB][4];
    auto slot4 = [&](int s, int b) {
      return reinterpret_cast<float4*>(base + static_cast<int64_t>(s) * na.Dp) + (lane + 32 * b);
    };
    // span row r = 2 (i - 1) (x) or 2 (i - 1) + 1 (p)
    auto span4 = [&](int r, int b) {
      return SMEM ? spans + r * (na.Dp / 4) + (lane + 32 * b) : slot4(kSlotSpan + r, b);
    };
    auto in_slot = [&](int b) { return 4 * (lane + 32 * b) < na.Dp; };
    auto put = [&](float4* q, const float (&v)[NB][4], int b) {
      *q = make_float4(v[b][0], v[b][1], v[b][2], v[b][3]);
    };
    auto get = [&](const float4* q, float (&v)[NB][4], int b) {
      const float4 w = *q;
      v[b][0] = w.x; v[b][1] = w.y; v[b][2] = w.z; v[b][3] = w.w;
    };
    auto store = [&](int s, const float (&v)[NB][4]) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (in_slot(b)) put(slot4(s, b), v, b);
    };
    auto load = [&](int s, float (&v)[NB][4]) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        v[b][0] = v[b][1] = v[b][2] = v[b][3] = 0.f;
        if (in_slot(b)) get(slot4(s, b), v, b);
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
    // both ends' U-turn tests: (dx . pa) < 0 or (dx . pb) < 0
    auto u_turn = [&](const float (&dx)[NB][4], const float (&pa)[NB][4], const float (&pb)[NB][4]) {
      float d1 = 0.f, d2 = 0.f;
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          d1 = fmaf(dx[b][i], pa[b][i], d1);
          d2 = fmaf(dx[b][i], pb[b][i], d2);
        }
      warp_sum2(d1, d2);
      return d1 < 0.f || d2 < 0.f;
    };
    const float half_n = 0.5f * static_cast<float>(D - 1);

    // The second half kick at the drifted x and every sum the leaf needs, in
    // one butterfly: log p (through the sum of squares), |p|^2 and, where
    // the span of two leaves closes here (close1), its U-turn dot products
    // dx . pf and dx . p with dx = sv (x - xf) against the span's first leaf
    // (xf, pf).  Sets g and p; returns log p, H = -log p + |p|^2 / 2 and
    // whether that span makes a U-turn.
    auto leaf_sums = [&](float h, float sv, bool close1, const float (&xf)[NB][4],
                         const float (&pf)[NB][4], float* H, bool* turn) {
      float q = 0.f, pp = 0.f, d1 = 0.f, d2 = 0.f;
      if (TARGET == HMC_T_STD_NORMAL) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            g[b][i] = -x[b][i];
            p[b][i] = fmaf(h, g[b][i], p[b][i]);
            q = fmaf(x[b][i], x[b][i], q);
            pp = fmaf(p[b][i], p[b][i], pp);
            const float dx = sv * (x[b][i] - xf[b][i]);
            d1 = fmaf(dx, pf[b][i], d1);
            d2 = fmaf(dx, p[b][i], d2);
          }
        warp_sum4(q, pp, d1, d2);
        const float lp = -0.5f * q;
        *H = -lp + 0.5f * pp;
        *turn = close1 && (d1 < 0.f || d2 < 0.f);
        return lp;
      } else {
        // funnel: dim 0 (lane 0, b 0, i 0) is v; its gradient needs the sum
        // of the others' squares, which the butterfly brings to every lane,
        // so its terms are added after it from broadcast copies
        const float v = __shfl_sync(0xffffffffu, x[0][0], 0);
        const float p0 = __shfl_sync(0xffffffffu, p[0][0], 0);
        const float xf0 = __shfl_sync(0xffffffffu, xf[0][0], 0);
        const float pf0 = __shfl_sync(0xffffffffu, pf[0][0], 0);
        const float ev = expf(-v);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const bool is_v = b == 0 && i == 0 && lane == 0;
            g[b][i] = -ev * x[b][i];
            if (!is_v) {
              p[b][i] = fmaf(h, g[b][i], p[b][i]);
              q = fmaf(x[b][i], x[b][i], q);
              pp = fmaf(p[b][i], p[b][i], pp);
              const float dx = sv * (x[b][i] - xf[b][i]);
              d1 = fmaf(dx, pf[b][i], d1);
              d2 = fmaf(dx, p[b][i], d2);
            }
          }
        warp_sum4(q, pp, d1, d2);
        const float g0 = v * (-1.f / 9.f) - half_n + 0.5f * ev * q;
        const float p0n = fmaf(h, g0, p0);
        if (lane == 0) {
          g[0][0] = g0;
          p[0][0] = p0n;
        }
        const float dx0 = sv * (v - xf0);
        d1 = fmaf(dx0, pf0, d1);
        d2 = fmaf(dx0, p0n, d2);
        const float lp = v * v * (-1.f / 18.f) - half_n * v - 0.5f * ev * q;
        *H = -lp + 0.5f * fmaf(p0n, p0n, pp);
        *turn = close1 && (d1 < 0.f || d2 < 0.f);
        return lp;
      }
    };

    // the chain's state at the start of the launch
    float lp = a.lp[c];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * (lane + 32 * b) + i;
        x[b][i] = d < D ? a.x[row + d] : 0.f;
        g[b][i] = d < D ? a.g[row + d] : 0.f;
      }
    unsigned long long leaves_total = 0ull;
    int moved = 0;
    for (int r = 0; r < na.T; ++r) {
      const long long t_full = a.t_full + r;
      const uint32_t t = static_cast<uint32_t>(t_full);
      // start: p0 ~ N(0, I), H0, log U
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = lane + 32 * b;
        const float4 z = momentum4(a.seed, static_cast<uint32_t>(j), chain, t);
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) p[b][i] = 4 * j + i < D ? zz[i] : 0.f;
      }
      const float H0 = -lp + 0.5f * dot(p, p);
      const float logU = accept_log_uniform(a.seed, chain, t);
      store(kSlotLeft, x); store(kSlotLeft + 1, p); store(kSlotLeft + 2, g);
      store(kSlotRight, x); store(kSlotRight + 1, p); store(kSlotRight + 2, g);
      store(kSlotCand, x); store(kSlotCand + 1, g);
      float lp_end[2] = {lp, lp};     // [0]: left, [1]: right
      float lpm = lp;
      uint32_t n = 1;
      moved = 0;
      float a_sum = 0.f;
      uint32_t n_a = 0;
      const uint32_t dirs = nuts_word0(a.seed, 0u, chain, t, kNutsTagDirection);
      for (int jd = 0; jd < na.max_depth; ++jd) {
        const int v = ((dirs >> jd) & 1u) ? 1 : -1;
        const float ev = static_cast<float>(v) * eps;
        const float hv = 0.5f * ev;
        const int side = v > 0 ? kSlotRight : kSlotLeft;
        load(side, x); load(side + 1, p); load(side + 2, g);
        lp = lp_end[v > 0 ? 1 : 0];
        uint32_t n_sub = 0;
        bool ok_sub = true;
        float lps = 0.f;
        const int leaves = 1 << jd;
        uint4 wsub4 = make_uint4(0u, 0u, 0u, 0u);
        for (int k = 0; k < leaves; ++k) {
          // the subtree-choice words depend on nothing the leaves compute:
          // drawn first, four at a time, the generator's arithmetic fills the
          // butterfly's latency
          if ((k & 3) == 0)
            wsub4 = philox(make_uint4(static_cast<uint32_t>(k >> 2), chain, t, kNutsTagSubtree + jd),
                           static_cast<uint32_t>(a.seed), static_cast<uint32_t>(a.seed >> 32));
          const int kq = k & 3;
          const uint32_t wsub = kq == 0 ? wsub4.x : kq == 1 ? wsub4.y : kq == 2 ? wsub4.z : wsub4.w;
          // spans of 2^i leaves closing at leaf k (2^i | k + 1); the span of
          // two leaves (i = 1) is tested inside the leaf's butterfly
          const int close = min(jd, __ffs(k + 1) - 1);
          float xf[NB][4], pf[NB][4];
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            xf[b][0] = xf[b][1] = xf[b][2] = xf[b][3] = 0.f;
            pf[b][0] = pf[b][1] = pf[b][2] = pf[b][3] = 0.f;
            if (close >= 1 && in_slot(b)) {
              get(span4(0, b), xf, b);
              get(span4(1, b), pf, b);
            }
          }
          // one leapfrog step of step v eps
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              p[b][i] = fmaf(hv, g[b][i], p[b][i]);
              x[b][i] = fmaf(ev, p[b][i], x[b][i]);
            }
          float H;
          bool turn;
          lp = leaf_sums(hv, static_cast<float>(v), close >= 1, xf, pf, &H, &turn);
          const bool finite = isfinite(H);
          if (!finite || H - H0 >= kNutsDeltaMax - logU) ok_sub = false;     // divergence
          a_sum += finite ? accept_prob(H0 - H) : 0.f;
          ++n_a;
          if (finite && logU <= H0 - H) {
            ++n_sub;
            if (nuts_take(wsub, 1u, n_sub)) {
              store(kSlotSub, x);
              store(kSlotSub + 1, g);
              lps = lp;
            }
          }
          if (turn) ok_sub = false;
          // spans of 2^i leaves opening at leaf k (2^i | k); no span both
          // opens and closes at one leaf
          const int open = k == 0 ? jd : min(jd, __ffs(k) - 1);
          for (int i = 1; i <= open; ++i) {
#pragma unroll
            for (int b = 0; b < NB; ++b)
              if (in_slot(b)) {
                put(span4(2 * (i - 1), b), x, b);
                put(span4(2 * (i - 1) + 1, b), p, b);
              }
          }
          for (int i = 2; i <= close && ok_sub; ++i) {
            float dx[NB][4], pg[NB][4];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              dx[b][0] = dx[b][1] = dx[b][2] = dx[b][3] = 0.f;
              pg[b][0] = pg[b][1] = pg[b][2] = pg[b][3] = 0.f;
              if (in_slot(b)) {
                get(span4(2 * (i - 1), b), dx, b);
                get(span4(2 * (i - 1) + 1, b), pg, b);
              }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
              for (int q = 0; q < 4; ++q) dx[b][q] = static_cast<float>(v) * (x[b][q] - dx[b][q]);
            if (u_turn(dx, pg, p)) ok_sub = false;
          }
          if (!ok_sub) break;
        }
        store(side, x); store(side + 1, p); store(side + 2, g);
        lp_end[v > 0 ? 1 : 0] = lp;
        if (!ok_sub) break;
        if (n_sub > 0 && nuts_take(nuts_word0(a.seed, static_cast<uint32_t>(jd), chain, t, kNutsTagTop), n_sub, n)) {
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
        if (u_turn(xr, pl, pr)) break;
      }
      // the new state
      load(kSlotCand, x);
      load(kSlotCand + 1, g);
      lp = lpm;
      prob = a_sum / static_cast<float>(n_a);
      leaves_total += n_a;
      const long long k = t_full - na.keep_from;
      if (k >= 0) {
        if (na.samples) {
          float* out = na.samples + k * CD + row;
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int d = 4 * (lane + 32 * b) + i;
              if (d < D) out[d] = x[b][i];
            }
        }
        if (lane == 0) {
          if (na.trace_acc) na.trace_acc[k * a.C + c] = static_cast<uint8_t>(moved);
          if (c == 0 && na.trace_eps) na.trace_eps[k] = eps;
        }
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * (lane + 32 * b) + i;
        if (d < D) {
          a.x[row + d] = x[b][i];
          a.g[row + d] = g[b][i];
        }
      }
    if (lane == 0) {
      a.lp[c] = lp;
      a.is_accepted[c] = static_cast<uint8_t>(moved);
      a.log_accept[c] = logf(prob);
      atomicAdd(na.leaves, leaves_total);
      atomicMax(na.leaves + 2, leaves_total);
    }
  }
  // the last transition's statistic (the only one that can adapt)
  const bool last = accept_tile_finish<kWarps>(a.da, a.partials, prob, has_chain, a.C, a.t_full + na.T - 1,
                                               static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
  // the launch lasts at least as long as its longest chain's leaves: the
  // critical path (the block that arrived last adds it)
  if (last && threadIdx.x == 0) {
    __threadfence();
    na.leaves[1] += atomicExch(na.leaves + 2, 0ull);
  }
}

template <int TARGET, int NB, bool SMEM>
cudaError_t launch_v(const NutsArgs& na, size_t smem, cudaStream_t s) {
  const unsigned grid = nuts_grid(na.s.C);
  k_nuts<TARGET, NB, SMEM><<<grid, 32 * kWarps, SMEM ? smem : 0, s>>>(na);
  count_launch();
  return cudaGetLastError();
}

template <int TARGET, int NB>
cudaError_t launch_nb(const NutsArgs& na, cudaStream_t s) {
  const size_t smem = span_smem_bytes(na.Dp, na.max_depth);
  // shared-memory span starts unless they cost resident chains: as many
  // blocks per SM as the scratch form, or enough for every chain
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorUnknown;
  }
  int occ_smem = 0, occ_glob = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ_glob, k_nuts<TARGET, NB, false>, 32 * kWarps, 0);
  if (e == cudaSuccess && smem <= kNutsSpanSmemMax)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_smem, k_nuts<TARGET, NB, true>,
                                                      32 * kWarps, smem);
  if (e != cudaSuccess) return e;
  const bool use_smem = smem > 0 && occ_smem > 0 &&
                        (occ_smem >= occ_glob ||
                         static_cast<int64_t>(occ_smem) * kWarps * sms >= na.s.C);
  return use_smem ? launch_v<TARGET, NB, true>(na, smem, s) : launch_v<TARGET, NB, false>(na, 0, s);
}

template <int TARGET>
cudaError_t launch_t(const NutsArgs& na, cudaStream_t s) {
  const int nb = (na.s.D + 127) / 128;
  if (nb <= 1) return launch_nb<TARGET, 1>(na, s);
  if (nb == 2) return launch_nb<TARGET, 2>(na, s);
  return launch_nb<TARGET, 4>(na, s);
}

template <int TARGET, int NB>
cudaError_t allow_smem() {
  return cudaFuncSetAttribute(k_nuts<TARGET, NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kNutsSpanSmemMax));
}

}  // namespace

bool nuts_supported(const hmc_target& t) {
  return (t.id == HMC_T_STD_NORMAL || t.id == HMC_T_FUNNEL) && t.dim <= kNutsMaxDim;
}

size_t nuts_scratch_floats(const hmc_target& t, int64_t C) {
  return static_cast<size_t>(C) * kNutsSlots * ((t.dim + 3) / 4 * 4);
}

unsigned nuts_grid(int64_t C) { return static_cast<unsigned>((C + kWarps - 1) / kWarps); }

cudaError_t nuts_prepare() {
  cudaError_t e = allow_smem<HMC_T_STD_NORMAL, 1>();
  if (e == cudaSuccess) e = allow_smem<HMC_T_STD_NORMAL, 2>();
  if (e == cudaSuccess) e = allow_smem<HMC_T_STD_NORMAL, 4>();
  if (e == cudaSuccess) e = allow_smem<HMC_T_FUNNEL, 1>();
  if (e == cudaSuccess) e = allow_smem<HMC_T_FUNNEL, 2>();
  if (e == cudaSuccess) e = allow_smem<HMC_T_FUNNEL, 4>();
  return e;
}

cudaError_t launch_nuts_transitions(const hmc_target& t, const StepArgs& a, float* scratch,
                                    int max_depth, unsigned long long* leaves, int T,
                                    long long keep_from, float* samples, float* trace_eps,
                                    uint8_t* trace_acc, cudaStream_t s, KernelTimer* timer) {
  NutsArgs na{a, scratch, (t.dim + 3) / 4 * 4, max_depth, leaves, T, keep_from, samples, trace_eps,
              trace_acc};
  if (timer) timer->begin(s);
  cudaError_t e = t.id == HMC_T_FUNNEL ? launch_t<HMC_T_FUNNEL>(na, s) : launch_t<HMC_T_STD_NORMAL>(na, s);
  if (timer) timer->end(s);
  return e;
}

cudaError_t launch_nuts_transition(const hmc_target& t, const StepArgs& a, float* scratch,
                                   int max_depth, unsigned long long* leaves, cudaStream_t s,
                                   KernelTimer* timer) {
  return launch_nuts_transitions(t, a, scratch, max_depth, leaves, 1, a.t_full, a.sample_out,
                                 a.trace_eps, a.trace_acc, s, timer);
}

}  // namespace hmc
