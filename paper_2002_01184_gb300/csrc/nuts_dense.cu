// The No-U-Turn Sampler (Section 2.3) for the dense targets -- the
// correlated Gaussian and the Bayesian logistic regression -- whose gradient
// is a matrix product over all chains (Section 2.1's batched evaluation).
//
// The transition and its random streams are those of the elementwise NUTS
// kernel (nuts.cu; Hoffman and Gelman's efficient NUTS with the recursion
// unrolled, O(max_depth) kept states).  What differs is the schedule: as in
// the paper's vectorised NUTS, the chains advance in lockstep, one leaf per
// iteration, with a mask for the chains whose trees have stopped.  One
// iteration is
//   (1) the batched gradient at every chain's drifted position: the 3xTF32
//       tcgen05 products of gauss_tc.cu (one-CTA tiles) or, for a logistic
//       regression of dim <= 128, logreg_tc.cu's CTA-pair kernel; a tile
//       whose chains have all stopped is skipped;
//   (2) one warp-per-chain kernel that finishes the leaf -- the gradient's
//       epilogue (sign, prior, split sum, log p), second half kick, energy,
//       slice and divergence tests, the candidate choice, the U-turn tests of
//       the spans that close, the subtree's and the trajectory's bookkeeping
//       -- and starts the next leaf (first half kick and drift of the chains
//       still building).
// For the logistic regression the iterations are the body of a CUDA-graph
// conditional WHILE node: the leaf kernel's last block clears the condition
// when no chain is left.  For the Gaussian the whole loop is one persistent
// cooperative launch (k_nuts_gauss_loop, below), products and leaves
// separated by bounded grid barriers.  Either way a transition costs as many
// iterations as its deepest tree and the host never waits on the device in
// between.  A chain's result depends only on its own row of every product,
// so it is the same in any batch.
//
// Per chain, the tree's scalars (NdChain) and a scratch of kNutsSlots rows of
// the padded row length (the two trajectory ends, the candidates, the span
// starts) stay in HBM between iterations; the working position is kept as its
// tf32 head and remainder -- the products' A operand -- and the momentum in the
// trajectory buffers of the tensor-core workspace.
#include <cmath>

#include <cuda.h>

#include "nuts_common.cuh"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

constexpr int kNdWarps = 8;

// the tree of one chain between iterations
struct NdChain {
  float H0, logU, lp_left, lp_right;
  float lpm, lps, lpw, a_sum;       // candidate, subtree candidate, working log p; sum of accept stats
  uint32_t dirs, n, n_sub, n_a;     // direction bits, valid leaves (tree, subtree), leaves built
  int j, k, active, moved;          // doubling, leaf in it, still building, candidate moved
};
static_assert(sizeof(NdChain) == 64, "chain record");

// products: gauss_tc.cu's tiles (Gaussian, logistic regression) or
// logreg_tc.cu's CTA pairs (logistic regression, dim <= 128); the last two
// share the leaf kernel
constexpr int kModeGauss = 0, kModeLogreg = 1, kModeLogregPair = 2;

struct NdArgs {
  StepArgs s;
  int ld;                 // row length of the working buffers and slots (D rounded up to 4)
  int max_depth;
  float* xhi;             // working position, tf32 head / remainder [C x ld]
  float* xlo;
  float* p;               // working momentum [C x ld]
  const float* part;      // products: X P, or the S partial sums of R X [S x C x ld]
  int S;                  // partial sums (logistic regression)
  const float* lp_part;   // logistic regression: log-likelihood partials, chain c's
  int nlp;                // nlp of them at lp_part[c * lp_cs + r * lp_rs]
  int64_t lp_cs, lp_rs;
  float* scratch;         // [C][kNutsSlots][ld]
  NdChain* st;
  uint8_t* active;
  unsigned* ctr;          // [0] chains left, [1] blocks arrived, [2] iterations of this transition
  int* err;
  unsigned long long* leaves;
  unsigned long long* iters;
  cudaGraphConditionalHandle handle;
};

template <int NB>
struct Lanes {
  const int lane;
  const int ld;
  __device__ bool ok(int b) const { return 4 * (lane + 32 * b) < ld; }
  __device__ float4* at(float* base, int64_t row, int b) const {
    return reinterpret_cast<float4*>(base + row) + (lane + 32 * b);
  }
  __device__ void put(float* base, int64_t row, const float (&v)[NB][4]) const {
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (ok(b)) *at(base, row, b) = make_float4(v[b][0], v[b][1], v[b][2], v[b][3]);
  }
  __device__ void get(const float* base, int64_t row, float (&v)[NB][4]) const {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ok(b)) w = *at(const_cast<float*>(base), row, b);
      v[b][0] = w.x; v[b][1] = w.y; v[b][2] = w.z; v[b][3] = w.w;
    }
  }
};

// (dx . pa) < 0 or (dx . pb) < 0
template <int NB>
__device__ __forceinline__ bool u_turn(const float (&dx)[NB][4], const float (&pa)[NB][4],
                                       const float (&pb)[NB][4]) {
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
}

// working position (x) and momentum (p) after the first half kick and the
// drift of a leaf of direction v: written for the next products
template <int NB>
__device__ __forceinline__ void half_kick_drift(const NdArgs& na, const Lanes<NB>& L, int64_t row, float hv,
                                                float ev, float (&x)[NB][4], float (&p)[NB][4],
                                                const float (&g)[NB][4]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      p[b][i] = fmaf(hv, g[b][i], p[b][i]);
      x[b][i] = fmaf(ev, p[b][i], x[b][i]);
      split_tf32(x[b][i], hi[i], lo[i]);
    }
    if (L.ok(b)) {
      *L.at(na.xhi, row, b) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *L.at(na.xlo, row, b) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      *L.at(na.p, row, b) = make_float4(p[b][0], p[b][1], p[b][2], p[b][3]);
    }
  }
}

__device__ __forceinline__ int dir_of(const NdChain& cs, int j) { return ((cs.dirs >> j) & 1u) ? 1 : -1; }

// Start of a transition (warp per chain): p0 ~ N(0, I), H0, log U, both
// trajectory ends and the candidate at the current state, then the first half
// kick and drift of leaf 0 of doubling 0.
template <int NB>
__global__ void __launch_bounds__(32 * kNdWarps) k_nuts_dense_begin(NdArgs na) {
  const StepArgs& a = na.s;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kNdWarps + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) na.ctr[2] = 0u;
  if (c >= a.C) return;
  const int D = a.D, ld = na.ld;
  const Lanes<NB> L{lane, ld};
  const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
  const float eps = a.da->eps;
  const int64_t srow = static_cast<int64_t>(c) * D;           // the state's rows have D floats
  const int64_t wrow = static_cast<int64_t>(c) * ld;
  float* base = na.scratch + static_cast<int64_t>(c) * kNutsSlots * ld;
  float x[NB][4], p[NB][4], g[NB][4];
  float pp = 0.f;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int q = lane + 32 * b;
    const float4 z = momentum4(a.seed, static_cast<uint32_t>(q), chain, a.t);
    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int d = 4 * q + i;
      const bool in = d < D;
      x[b][i] = in ? a.x[srow + d] : 0.f;
      g[b][i] = in ? a.g[srow + d] : 0.f;
      p[b][i] = in ? zz[i] : 0.f;
      pp = fmaf(p[b][i], p[b][i], pp);
    }
  }
  pp = warp_sum(pp);
  const float lp = a.lp[c];
  NdChain cs;
  cs.H0 = -lp + 0.5f * pp;
  cs.logU = accept_log_uniform(a.seed, chain, a.t);
  cs.lp_left = cs.lp_right = cs.lpm = cs.lpw = lp;
  cs.lps = 0.f;
  cs.a_sum = 0.f;
  cs.dirs = nuts_word0(a.seed, 0u, chain, a.t, kNutsTagDirection);
  cs.n = 1u;
  cs.n_sub = cs.n_a = 0u;
  cs.j = cs.k = 0;
  cs.active = 1;
  cs.moved = 0;
  L.put(base, kSlotLeft * ld, x);
  L.put(base, (kSlotLeft + 1) * ld, p);
  L.put(base, (kSlotLeft + 2) * ld, g);
  L.put(base, kSlotRight * ld, x);
  L.put(base, (kSlotRight + 1) * ld, p);
  L.put(base, (kSlotRight + 2) * ld, g);
  L.put(base, kSlotCand * ld, x);
  L.put(base, (kSlotCand + 1) * ld, g);
  const float ev = static_cast<float>(dir_of(cs, 0)) * eps;
  half_kick_drift(na, L, wrow, 0.5f * ev, ev, x, p, g);
  if (lane == 0) {
    na.st[c] = cs;
    na.active[c] = 1;
  }
}

// One leaf of chain c (active, its gradient products done; the whole warp):
// returns whether the chain is still building its tree.
template <int MODE, int NB>
__device__ __forceinline__ bool nuts_leaf(const NdArgs& na, int c, int lane) {
  const StepArgs& a = na.s;
  bool still = false;
  {
    NdChain cs = na.st[c];
    const int D = a.D, ld = na.ld;
    const Lanes<NB> L{lane, ld};
    const int64_t row = static_cast<int64_t>(c) * ld;
    const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
    const uint32_t t = a.t;
    const float eps = a.da->eps;
    float* base = na.scratch + static_cast<int64_t>(c) * kNutsSlots * ld;
    auto slot = [&](int s) { return static_cast<int64_t>(s) * ld; };
    int v = dir_of(cs, cs.j);
    float hv = 0.5f * static_cast<float>(v) * eps;
    // spans of 2^i leaves closing here (2^i | k + 1); the first one's start
    // is read before the butterfly so that its U-turn sums join it
    const int close = min(cs.j, __ffs(cs.k + 1) - 1);
    float x[NB][4], p[NB][4], g[NB][4], xf[NB][4], pf[NB][4];
    {
      float hi[NB][4], lo[NB][4];
      L.get(na.xhi, row, hi);
      L.get(na.xlo, row, lo);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) x[b][i] = hi[b][i] + lo[b][i];
    }
    L.get(na.p, row, p);
    if (close >= 1) {
      L.get(base, slot(kSlotSpan), xf);
      L.get(base, slot(kSlotSpan + 1), pf);
    } else {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < 4; ++i) xf[b][i] = pf[b][i] = 0.f;
    }
    // the gradient at x from the products, the second half kick, and the sums
    float s0 = 0.f, pp = 0.f, d1 = 0.f, d2 = 0.f;
    const int64_t split = static_cast<int64_t>(a.C) * ld;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (L.ok(b)) {
        const float4* pr = reinterpret_cast<const float4*>(na.part + row) + (lane + 32 * b);
        gv = *pr;
        if (MODE == kModeLogreg)
          for (int sp = 1; sp < na.S; ++sp) {
            const float4 u = pr[sp * (split / 4)];
            gv.x += u.x; gv.y += u.y; gv.z += u.z; gv.w += u.w;
          }
      }
      const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * (lane + 32 * b) + i;
        // Gaussian: g = -x P; logistic regression: g = R X - theta (the
        // N(0, I) prior), zero on the padding
        g[b][i] = MODE == kModeGauss ? -gg[i] : (d < D ? gg[i] - x[b][i] : 0.f);
        p[b][i] = fmaf(hv, g[b][i], p[b][i]);
        s0 = MODE == kModeGauss ? fmaf(x[b][i], g[b][i], s0) : fmaf(x[b][i], x[b][i], s0);
        pp = fmaf(p[b][i], p[b][i], pp);
        const float dx = static_cast<float>(v) * (x[b][i] - xf[b][i]);
        d1 = fmaf(dx, pf[b][i], d1);
        d2 = fmaf(dx, p[b][i], d2);
      }
    }
    float rows = 0.f;
    if (MODE == kModeLogreg) {
      for (int r = lane; r < na.nlp; r += 32) rows += na.lp_part[c * na.lp_cs + r * na.lp_rs];
      rows = warp_sum(rows);
    }
    warp_sum4(s0, pp, d1, d2);
    // Gaussian: log p = <x, g> / 2; logistic regression: the rows'
    // log-likelihood minus |theta|^2 / 2
    const float lp = MODE == kModeGauss ? 0.5f * s0 : rows - 0.5f * s0;
    const float H = -lp + 0.5f * pp;
    bool ok = true;
    const bool finite = isfinite(H);
    if (!finite || H - cs.H0 >= kNutsDeltaMax - cs.logU) ok = false;       // divergence
    cs.a_sum += finite ? accept_prob(cs.H0 - H) : 0.f;
    cs.n_a += 1u;
    if (finite && cs.logU <= cs.H0 - H) {
      cs.n_sub += 1u;
      if (nuts_take(nuts_subtree_word(a.seed, static_cast<uint32_t>(cs.k), chain, t, cs.j), 1u, cs.n_sub)) {
        L.put(base, slot(kSlotSub), x);
        L.put(base, slot(kSlotSub + 1), g);
        cs.lps = lp;
      }
    }
    if (close >= 1 && (d1 < 0.f || d2 < 0.f)) ok = false;
    for (int i = 2; i <= close && ok; ++i) {
      float xs[NB][4], ps[NB][4];
      L.get(base, slot(kSlotSpan + 2 * (i - 1)), xs);
      L.get(base, slot(kSlotSpan + 2 * (i - 1) + 1), ps);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) xs[b][q] = static_cast<float>(v) * (x[b][q] - xs[b][q]);
      if (u_turn(xs, ps, p)) ok = false;
    }
    if (ok) {
      // spans of 2^i leaves opening here (2^i | k); none opens and closes at one leaf
      const int open = cs.k == 0 ? cs.j : min(cs.j, __ffs(cs.k) - 1);
      for (int i = 1; i <= open; ++i) {
        L.put(base, slot(kSlotSpan + 2 * (i - 1)), x);
        L.put(base, slot(kSlotSpan + 2 * (i - 1) + 1), p);
      }
    }
    cs.lpw = lp;
    bool done = !ok;
    if (ok && cs.k + 1 == (1 << cs.j)) {
      // the subtree is complete: it becomes the trajectory's end on its side
      const int side = v > 0 ? kSlotRight : kSlotLeft;
      L.put(base, slot(side), x);
      L.put(base, slot(side + 1), p);
      L.put(base, slot(side + 2), g);
      if (v > 0) cs.lp_right = lp;
      else cs.lp_left = lp;
      if (cs.n_sub > 0u &&
          nuts_take(nuts_word0(a.seed, static_cast<uint32_t>(cs.j), chain, t, kNutsTagTop), cs.n_sub, cs.n)) {
        float t1[NB][4], t2[NB][4];
        L.get(base, slot(kSlotSub), t1);
        L.get(base, slot(kSlotSub + 1), t2);
        L.put(base, slot(kSlotCand), t1);
        L.put(base, slot(kSlotCand + 1), t2);
        cs.lpm = cs.lps;
        cs.moved = 1;
      }
      cs.n += cs.n_sub;
      // the whole trajectory's ends
      float xl[NB][4], pl[NB][4], xr[NB][4], pr[NB][4];
      L.get(base, slot(kSlotLeft), xl);
      L.get(base, slot(kSlotLeft + 1), pl);
      L.get(base, slot(kSlotRight), xr);
      L.get(base, slot(kSlotRight + 1), pr);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) xr[b][q] -= xl[b][q];
      if (u_turn(xr, pl, pr) || cs.j + 1 >= na.max_depth) {
        done = true;
      } else {
        // next doubling: grow from the end on its side
        cs.j += 1;
        cs.k = 0;
        cs.n_sub = 0u;
        v = dir_of(cs, cs.j);
        const int from = v > 0 ? kSlotRight : kSlotLeft;
        L.get(base, slot(from), x);
        L.get(base, slot(from + 1), p);
        L.get(base, slot(from + 2), g);
        cs.lpw = v > 0 ? cs.lp_right : cs.lp_left;
      }
    } else if (ok) {
      cs.k += 1;
    }
    if (done) {
      cs.active = 0;
    } else {
      const float ev = static_cast<float>(v) * eps;
      half_kick_drift(na, L, row, 0.5f * ev, ev, x, p, g);
      still = true;
    }
    if (lane == 0) {
      na.st[c] = cs;
      na.active[c] = still ? 1 : 0;
    }
  }
  return still;
}

// One leaf of every chain still building its tree, then the loop condition.
template <int MODE, int NB>
__global__ void __launch_bounds__(32 * kNdWarps) k_nuts_dense_leaf(NdArgs na) {
  const StepArgs& a = na.s;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kNdWarps + (threadIdx.x >> 5);
  bool still = false;
  if (c < a.C && na.st[c].active) still = nuts_leaf<MODE, NB>(na, c, lane);
  // the loop condition: any chain left (the last block to arrive decides);
  // a tree has at most 2^max_depth - 1 leaves, so more iterations than that
  // mean a fault of the bookkeeping: the loop stops and the flag reports it
  const int left = __syncthreads_count((threadIdx.x & 31) == 0 && still);
  if (threadIdx.x == 0) {
    if (left) atomicAdd(&na.ctr[0], static_cast<unsigned>(left));
    __threadfence();
    const unsigned prev = atomicAdd(&na.ctr[1], 1u);
    if (prev == gridDim.x - 1u) {
      __threadfence();
      const unsigned total = atomicAdd(&na.ctr[0], 0u);
      const unsigned it = na.ctr[2] + 1u;
      bool more = total > 0u;
      if (more && it >= (1u << na.max_depth)) {
        more = false;
        atomicExch(na.err, 2);
      }
      na.ctr[0] = 0u;
      na.ctr[1] = 0u;
      na.ctr[2] = it;
      *na.iters += 1ull;
      __threadfence();
      cudaGraphSetConditional(na.handle, more ? 1u : 0u);
    }
  }
}

// End of a transition (warp per chain): the candidate becomes the state;
// kernel results, kept sample, traces, leaf count; the acceptance statistic
// (mean over the leaves built) enters dual averaging.
__global__ void __launch_bounds__(32 * kNdWarps) k_nuts_dense_finish(NdArgs na) {
  const StepArgs& a = na.s;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kNdWarps + (threadIdx.x >> 5);
  const bool has = c < a.C;
  const float eps = a.da->eps;
  float prob = 0.f;
  unsigned n_a = 0u;
  if (has) {
    const NdChain cs = na.st[c];
    const int D = a.D, ld = na.ld;
    const float* base = na.scratch + static_cast<int64_t>(c) * kNutsSlots * ld;
    const int64_t srow = static_cast<int64_t>(c) * D;
    for (int d = lane; d < D; d += 32) {
      const float xv = base[kSlotCand * ld + d];
      a.x[srow + d] = xv;
      a.g[srow + d] = base[(kSlotCand + 1) * ld + d];
      if (a.sample_out) a.sample_out[srow + d] = xv;
    }
    prob = cs.a_sum / static_cast<float>(cs.n_a);
    n_a = cs.n_a;
    if (lane == 0) {
      a.lp[c] = cs.lpm;
      a.is_accepted[c] = static_cast<uint8_t>(cs.moved);
      a.log_accept[c] = logf(prob);
      if (a.trace_acc) a.trace_acc[c] = static_cast<uint8_t>(cs.moved);
      if (c == 0 && a.trace_eps) a.trace_eps[0] = eps;
    }
  }
  __shared__ unsigned long long blk_leaves;
  if (threadIdx.x == 0) blk_leaves = 0ull;
  __syncthreads();
  if (has && lane == 0) atomicAdd(&blk_leaves, static_cast<unsigned long long>(n_a));
  __syncthreads();
  if (threadIdx.x == 0 && blk_leaves) atomicAdd(na.leaves, blk_leaves);
  accept_tile_finish<kNdWarps>(a.da, a.partials, prob, has, a.C, a.t_full, static_cast<int>(blockIdx.x),
                               static_cast<int>(gridDim.x));
}

// ---- the dense Gaussian's leaf loop in one persistent cooperative launch
//
// The graph loop above pays two kernel launches, the products' set-up
// (barriers, tensor memory) and the WHILE node's relaunch every leaf: about
// 15 us whatever the size.  For the Gaussian the whole loop runs instead in
// one cooperative launch of one CTA per SM: each iteration is the tile
// products X P of the 128-chain tiles still building (3xTF32 tcgen05, 64
// output dims per tile, tiles dealt round-robin to the CTAs; the pipeline's
// barriers and tensor memory set up once), a grid barrier, the leaf of every
// active chain (warp per chain over all warps of the grid), and a second
// grid barrier that also counts the chains left.  Grid barriers are bounded
// (a wait that gives up sets the error flag and every CTA leaves the loop).
constexpr int kPlBM = 128, kPlBN = 64, kPlBK = 32, kPlStages = 4;
constexpr int kPlWarps = 18;                         // 0 TMA, 1 MMA, 2-17 epilogue (all 18: leaves)
constexpr int kPlThreads = 32 * kPlWarps;
constexpr uint32_t kPlABytes = kPlBM * kPlBK * 4;    // 16 KB: 128 chains x 32 dims
constexpr uint32_t kPlBBytes = kPlBN * kPlBK * 4;    // 8 KB: 64 rows of P x 32 dims
constexpr uint32_t kPlStage = 2 * kPlABytes + 2 * kPlBBytes;
// ring + alignment slack + barriers (10 x 8 B), tensor-memory slot (16 B),
// the tile list (kPlMaxTiles ints) and two flags
constexpr size_t kPlSmem = kPlStages * kPlStage + 1024 + 512;
constexpr int kPlMaxTiles = 64;                      // tiles of one CTA per iteration (the host checks)
static_assert(10 * 8 + 16 + 4 * kPlMaxTiles + 8 <= 512, "small shared-memory area");

__device__ __forceinline__ bool pl_grid_barrier(unsigned* counter, unsigned gen) {
  __threadfence();
  atomicAdd(counter, 1u);
  const unsigned target = gen * gridDim.x;
  const unsigned long long t0 = ptx::global_timer_ns();
  while (*reinterpret_cast<volatile unsigned*>(counter) < target) {
    if (ptx::global_timer_ns() - t0 > ptx::kWaitLimitNs) return false;
  }
  __threadfence();
  return true;
}

template <int NB>
__global__ void __launch_bounds__(kPlThreads, 1)
k_nuts_gauss_loop(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                  const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                  NdArgs na) {
  const StepArgs& a = na.s;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPlStages * kPlStage);
  uint64_t* empty = full + kPlStages;
  uint64_t* acc_full = empty + kPlStages;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  int* tile_id = reinterpret_cast<int*>(tmem_slot + 4);       // [kPlMaxTiles] this iteration's tiles
  int* flags = tile_id + kPlMaxTiles;                          // [0] tiles, [1] leave the loop

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = a.C, D = a.D;
  const int nk = (D + kPlBK - 1) / kPlBK;
  const int mt = (C + kPlBM - 1) / kPlBM, ntn = (D + kPlBN - 1) / kPlBN;
  const int ntiles = mt * ntn;
  unsigned* bar = na.ctr + 3;            // grid barrier counter (zeroed before the launch)
  unsigned* left = na.ctr + 4;           // [2] chains left, by iteration parity

  if (threadIdx.x == 0) {
    for (int i = 0; i < kPlStages; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&empty[i], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(acc_empty, 32 * (kPlWarps - 2));
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mAhi);
    ptx::prefetch_tensormap(&mAlo);
    ptx::prefetch_tensormap(&mBhi);
    ptx::prefetch_tensormap(&mBlo);
    flags[1] = 0;
  }
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kPlBN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // pipeline positions, kept by the thread of each role across iterations
  int pit = 0;          // producer: stages filled
  int mit = 0;          // issuer: stages consumed
  int mtile = 0;        // issuer: tiles committed
  int etile = 0;        // epilogue: tiles drained
  unsigned gen = 0;     // grid barriers met
  const int gwarps = static_cast<int>(gridDim.x) * kPlWarps;
  const int gw = static_cast<int>(blockIdx.x) * kPlWarps + warp;
  for (int it = 0;; ++it) {
    // ---- this CTA's tiles with an active chain (tiles blockIdx.x + k gridDim.x)
    if (threadIdx.x == 0) flags[0] = 0;
    __syncthreads();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int m0 = (t / ntn) * kPlBM;
      const int r = threadIdx.x;
      const bool mine = r < kPlBM && m0 + r < C && na.active[m0 + r] != 0;
      if (__syncthreads_or(mine) && threadIdx.x == 0 && flags[0] < kPlMaxTiles) tile_id[flags[0]++] = t;
    }
    __syncthreads();
    const int nt = flags[0];
    if (warp == 0 && lane == 0) {
      // ---- TMA producer: x (head / remainder) of the tile's 128 chains, 64 rows of P
      for (int k = 0; k < nt; ++k) {
        const int t = tile_id[k];
        const int m0 = (t / ntn) * kPlBM, n0 = (t % ntn) * kPlBN;
        for (int kc = 0; kc < nk; ++kc, ++pit) {
          const int st = pit % kPlStages, round = pit / kPlStages;
          if (pit >= kPlStages && !ptx::mbar_wait(&empty[st], (round - 1) & 1)) {
            atomicExch(na.err, 1);
            break;
          }
          uint8_t* sp = smem + st * kPlStage;
          ptx::mbar_arrive_expect_tx(&full[st], kPlStage);
          const int kx = kc * kPlBK;
          ptx::tma_load_2d(sp, &mAhi, &full[st], kx, m0);
          ptx::tma_load_2d(sp + kPlABytes, &mAlo, &full[st], kx, m0);
          ptx::tma_load_2d(sp + 2 * kPlABytes, &mBhi, &full[st], kx, n0);
          ptx::tma_load_2d(sp + 2 * kPlABytes + kPlBBytes, &mBlo, &full[st], kx, n0);
        }
      }
    } else if (warp == 1 && lane == 0) {
      // ---- MMA issuer: 3xTF32, A_lo B_hi + A_hi B_lo + A_hi B_hi
      constexpr uint32_t idesc = ptx::idesc_tf32(kPlBM, kPlBN);
      for (int k = 0; k < nt; ++k, ++mtile) {
        // the accumulator is free once the previous tile's epilogue read it
        if (mtile > 0 && !ptx::mbar_wait(acc_empty, (mtile - 1) & 1)) atomicExch(na.err, 1);
        ptx::tc_fence_after();
        for (int kc = 0; kc < nk; ++kc, ++mit) {
          const int st = mit % kPlStages, round = mit / kPlStages;
          if (!ptx::mbar_wait(&full[st], round & 1)) {
            atomicExch(na.err, 1);
            break;
          }
          ptx::tc_fence_after();
          const uint32_t sp = ptx::smem_u32(smem + st * kPlStage);
#pragma unroll
          for (int j = 0; j < kPlBK / 8; ++j) {
            const uint64_t a_hi = ptx::sw128_kmajor_desc(sp + 32 * j);
            const uint64_t a_lo = ptx::sw128_kmajor_desc(sp + kPlABytes + 32 * j);
            const uint64_t b_hi = ptx::sw128_kmajor_desc(sp + 2 * kPlABytes + 32 * j);
            const uint64_t b_lo = ptx::sw128_kmajor_desc(sp + 2 * kPlABytes + kPlBBytes + 32 * j);
            ptx::mma_tf32(tmem, a_lo, b_hi, idesc, (kc | j) != 0 ? 1u : 0u);
            ptx::mma_tf32(tmem, a_hi, b_lo, idesc, 1u);
            ptx::mma_tf32(tmem, a_hi, b_hi, idesc, 1u);
          }
          ptx::mma_commit(&empty[st]);
        }
        ptx::mma_commit(acc_full);
      }
    } else if (warp >= 2) {
      // ---- epilogue: warp (quarter q, column group g) stores X P for rows
      // 32 q .. 32 q + 31 of the tile, columns 16 g .. 16 g + 15, each lane
      // one row (64 contiguous bytes)
      const int quarter = warp & 3, cg = (warp - 2) >> 2;
      for (int k = 0; k < nt; ++k, ++etile) {
        const int t = tile_id[k];
        const int m0 = (t / ntn) * kPlBM, n0 = (t % ntn) * kPlBN;
        if (!ptx::mbar_wait(acc_full, etile & 1)) atomicExch(na.err, 1);
        ptx::tc_fence_after();
        float v[16];
        ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + 16 * cg, v);
        ptx::tc_fence_before();
        ptx::mbar_arrive_local(acc_empty);
        const int m = m0 + quarter * 32 + lane;
        const int n = n0 + 16 * cg;
        if (m < C) {
          // D % 4 == 0 on this path: a float4 lies wholly inside or past the row
          float4* out = reinterpret_cast<float4*>(const_cast<float*>(na.part) + static_cast<int64_t>(m) * D + n);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (n + 4 * q < D) out[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
    }
    // ---- the products are in: every CTA's leaves may read them (the CTA
    // barrier, then thread 0's fence in the grid barrier, publish every
    // thread's stores, as a grid-wide sync does)
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!pl_grid_barrier(bar, ++gen)) {
        atomicExch(na.err, 3);
        flags[1] = 1;
      }
      if (blockIdx.x == 0) left[(it + 1) & 1] = 0u;     // the slot the next iteration counts in
    }
    __syncthreads();
    if (flags[1]) break;
    // ---- one leaf of every active chain
    int mine = 0;
    for (int c = gw; c < C; c += gwarps)
      if (na.st[c].active && nuts_leaf<kModeGauss, NB>(na, c, lane)) ++mine;
    // positions written for the next products' TMA loads (another proxy)
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (lane == 0 && mine) atomicAdd(&left[it & 1], static_cast<unsigned>(mine));
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!pl_grid_barrier(bar, ++gen)) {
        atomicExch(na.err, 3);
        flags[1] = 1;
      } else {
        const unsigned total = *reinterpret_cast<volatile unsigned*>(&left[it & 1]);
        if (blockIdx.x == 0) *na.iters += 1ull;
        if (total == 0u) {
          flags[1] = 1;
        } else if (it + 1 >= (1 << na.max_depth)) {
          if (blockIdx.x == 0) atomicExch(na.err, 2);
          flags[1] = 1;
        }
      }
    }
    __syncthreads();
    if (flags[1]) break;
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kPlBN);
  }
}

template <int NB>
cudaError_t set_leaf_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_nuts_dense_leaf<kModeGauss, NB>,
                                       cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nuts_dense_leaf<kModeLogreg, NB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             0);
  return e;
}

// CTAs of the Gaussian's persistent leaf loop for C chains, 0 if it does not
// apply (every CTA's tiles must fit its list, all CTAs resident at once)
int gauss_loop_grid(int C, int D, int* sms_out = nullptr) {
  static int sms = 0, occ = -1;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  if (occ < 0) {
    int o = 0;
    const int nb = (D + 3) / 4 * 4 <= 128 ? 1 : (D + 3) / 4 * 4 <= 256 ? 2 : 4;
    cudaError_t e = nb == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nuts_gauss_loop<1>, kPlThreads, kPlSmem)
                  : nb == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nuts_gauss_loop<2>, kPlThreads, kPlSmem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nuts_gauss_loop<4>, kPlThreads, kPlSmem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    occ = o;
  }
  if (occ < 1) return 0;
  if (sms_out) *sms_out = sms;
  const int ntiles = ((C + kPlBM - 1) / kPlBM) * ((D + kPlBN - 1) / kPlBN);
  const int want = std::max(ntiles, (C + kPlWarps - 1) / kPlWarps);
  const int grid = std::min(sms * occ, want);
  if (static_cast<int64_t>(grid) * kPlMaxTiles < ntiles) return 0;
  return grid;
}

template <int NB>
cudaError_t enqueue_nb(const hmc_target& t, const NdArgs& base_args, NutsDense& nd, cudaStream_t s,
                       KernelTimer* timer) {
  const StepArgs& a = base_args.s;
  const unsigned nb = static_cast<unsigned>((a.C + kNdWarps - 1) / kNdWarps);
  NdArgs na = base_args;
  if (timer) timer->begin(s);
  k_nuts_dense_begin<NB><<<nb, 32 * kNdWarps, 0, s>>>(na);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int pgrid = nd.mode == kModeGauss ? gauss_loop_grid(a.C, a.D) : 0;
  if (pgrid > 0) {
    // the whole leaf loop in one cooperative launch (grid barrier and the
    // two chains-left counters zeroed first)
    e = cudaMemsetAsync(nd.ctr + 3, 0, 3 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(pgrid));
    cfg.blockDim = dim3(kPlThreads);
    cfg.dynamicSmemBytes = kPlSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GaussTc& tc = *nd.tc;
    e = cudaLaunchKernelEx(&cfg, k_nuts_gauss_loop<NB>, tc.mAhi[0], tc.mAlo[0], tc.mBhi, tc.mBlo, na);
    count_launch();
    if (e != cudaSuccess) return e;
    k_nuts_dense_finish<<<nb, 32 * kNdWarps, 0, s>>>(na);
    count_launch();
    if (timer) timer->end(s);
    return cudaGetLastError();
  }
  // the leaf loop: a WHILE node after everything captured so far
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureImplicit;
  cudaGraphConditionalHandle handle = 0;
  e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  // the body: products, then the leaf kernel
  e = cudaStreamBeginCaptureToGraph(nd.side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  na.handle = handle;
  if (nd.mode == kModeGauss) {
    e = launch_gauss_tc_product(*nd.tc, a.C, a.D, a.da, nd.active, nd.side);
  } else if (nd.mode == kModeLogreg) {
    int S = 1;
    e = launch_logreg_gemm_products(*nd.lrg, a.C, a.D, a.da, nd.active, &S, nd.side);
    na.S = S;
  } else {     // kModeLogregPair
    e = launch_logreg_tc_grad(*nd.lrtc, a.C, a.D, nd.active, nd.err, nd.side);
  }
  if (e == cudaSuccess) {
    if (nd.mode == kModeGauss)
      k_nuts_dense_leaf<kModeGauss, NB><<<nb, 32 * kNdWarps, 0, nd.side>>>(na);
    // (both logistic-regression product forms leave S partial sums)
    else
      k_nuts_dense_leaf<kModeLogreg, NB><<<nb, 32 * kNdWarps, 0, nd.side>>>(na);
    count_launch();
    e = cudaGetLastError();
  }
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(nd.side, &captured);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  k_nuts_dense_finish<<<nb, 32 * kNdWarps, 0, s>>>(na);
  count_launch();
  if (timer) timer->end(s);
  return cudaGetLastError();
}

}  // namespace

bool nuts_dense_supported(const hmc_target& t) {
  if (t.dim > kNutsMaxDim) return false;
  return (t.id == HMC_T_CORR_GAUSS && gauss_tc_supported(t)) ||
         (t.id == HMC_T_LOGREG && (logreg_tc_supported(t) || logreg_gemm_supported(t)));
}

size_t nuts_dense_chain_bytes(int64_t C) { return static_cast<size_t>(C) * sizeof(NdChain); }

cudaError_t nuts_dense_prepare() {
  cudaError_t e = set_leaf_attrs<1>();
  if (e == cudaSuccess) e = set_leaf_attrs<2>();
  if (e == cudaSuccess) e = set_leaf_attrs<4>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nuts_gauss_loop<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kPlSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nuts_gauss_loop<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kPlSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nuts_gauss_loop<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kPlSmem));
  return e;
}

cudaError_t launch_nuts_dense_transition(const hmc_target& t, const StepArgs& a, NutsDense& nd, cudaStream_t s,
                                         KernelTimer* timer) {
  if (nd.mode != kModeGauss && nd.mode != kModeLogreg && nd.mode != kModeLogregPair) return cudaErrorInvalidValue;
  NdArgs na{};
  na.s = a;
  na.ld = (t.dim + 3) / 4 * 4;
  na.max_depth = nd.max_depth;
  na.S = 1;
  if (nd.mode == kModeGauss) {
    na.xhi = nd.tc->xhi[0];
    na.xlo = nd.tc->xlo[0];
    na.p = nd.tc->p;
    na.part = nd.tc->gL;
  } else if (nd.mode == kModeLogreg) {
    // (S is set when the products are enqueued)
    na.xhi = nd.lrg->xhi[0];
    na.xlo = nd.lrg->xlo[0];
    na.p = nd.lrg->p;
    na.part = nd.lrg->part;
    na.lp_part = nd.lrg->lp_part;
    na.nlp = nd.lrg->nrt;             // the row tiles' columns of [C x ntot]
    na.lp_cs = nd.lrg->ntot;
    na.lp_rs = 1;
  } else {
    na.xhi = nd.lrtc->thi;
    na.xlo = nd.lrtc->tlo;
    na.p = nd.lrtc->p;
    na.part = nd.lrtc->Gpart;
    na.S = nd.lrtc->nsplit;
    na.lp_part = nd.lrtc->lp_part;
    na.nlp = nd.lrtc->nsplit;         // [nsplit x C]
    na.lp_cs = 1;
    na.lp_rs = a.C;
  }
  na.scratch = nd.scratch;
  na.st = static_cast<NdChain*>(nd.chains);
  na.active = nd.active;
  na.ctr = nd.ctr;
  na.err = nd.err;
  na.leaves = nd.leaves;
  na.iters = nd.iters;
  const int nb = (na.ld + 127) / 128;
  if (nb <= 1) return enqueue_nb<1>(t, na, nd, s, timer);
  if (nb == 2) return enqueue_nb<2>(t, na, nd, s, timer);
  return enqueue_nb<4>(t, na, nd, s, timer);
}

}  // namespace hmc
