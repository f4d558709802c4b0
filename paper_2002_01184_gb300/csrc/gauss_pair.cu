// HMC transitions for the dense Gaussian target (dim <= 256) on CTA pairs
// (tcgen05 cta_group::2).  A pair owns 64 chains; one launch runs T
// consecutive transitions of them (Section 2.1's transition, Section 4.2's
// driver loop), so that P stays resident across transitions and no launch
// sits between them.  Each leapfrog gradient G^T = P X^T (3xTF32) is one
// stream of M = 256 (all output dims) MMAs issued by the pair's leader, two
// per K-step of 8 dims:
//   * B (positions) stacks each CTA's 32 chains' tf32 heads and remainders
//     as 64 rows of one 128-byte-swizzled K-major tile, so one N = 128 MMA
//     with A = P head forms P_hi x_hi and P_hi x_lo for all 64 chains, and
//     one N = 64 MMA with A = P remainder over the head rows alone adds
//     P_lo x_hi -- two instructions where three separate products of N = 64
//     took three (the MMAs are bound by their issue rate at this N).
//   * Accumulators (128 tensor-memory columns): column (CTA q, row r) of the
//     N = 128 product; the N = 64 product is written at column offset 32, so
//     that each chain's P_lo x_hi lands in one of its own two columns.  A
//     chain's gradient is the sum of its two columns.
//   * A (P head / remainder) is resident for the whole launch: each CTA's 128
//     rows of P, the head of every K-chunk and the remainder of K-chunks 0-3
//     in its tensor memory, the remainder of K-chunks 4-7 in shared memory
//     (A operands read from shared memory slow the MMAs down more for the
//     N = 128 product than for the N = 64 one).
//   * Epilogue (warps 2-9 of both CTAs): one output dim per thread and 32
//     chains per thread, 16 of the peer's and 16 of its own; momenta and
//     trajectory positions in registers, the chains' current positions (this
//     CTA's dims) in shared memory and their cached gradients in global
//     memory (L2) across transitions.  Each step a thread first updates its
//     peer chains, whose next positions are staged locally (in the
//     destination's layout); each warp then pushes its 16 rows of a K-chunk
//     (head and remainder, 2 KB each) to the peer by bulk DSMEM copy,
//     completing on the peer's tile barrier, and updates its own chains,
//     written straight into its tile, while the copy is in flight.
//   * Readiness is tracked per half of K: in each CTA's tile the K-chunks of
//     its own dims are written locally (own_full, which every epilogue thread
//     joins once it has read the accumulators) and the other four arrive by
//     copy (in_full).  The peer forwards both completions to the leader.  The
//     issuer starts on K-chunks 4-7, whose leader half arrives by copy
//     straight onto the leader's barrier, and reaches K-chunks 0-3, whose
//     peer half needs the copy plus the forward, a quarter-step of MMAs later.
//   * The momenta of the next transition are drawn while the epilogue waits
//     for the MMAs (counter-based, so the draw order is free) and parked in
//     global memory, in per-thread float4 blocks; the cached gradients of
//     the launch live in such blocks too.
// Both CTAs form H_L and decide every chain of the pair from their two
// partial sums; each CTA writes its kept sample as one tensor store.  With
// T > 1 the launch is cooperative: after every transition that adapts the
// step size (and after the last one) all CTAs meet at a grid barrier that
// also sums the fixed-point acceptance statistic, and each applies the same
// dual-averaging update to its own copy of the state; a launch of one
// transition instead lets its last CTA update the state.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

constexpr int kMaxDim = 256;
constexpr int kChunks = kMaxDim / 32;             // K-chunks of 32 dims
constexpr int kLoTmemChunks = 4;                  // P remainder chunks held in tensor memory
constexpr int kHalfChunks = kChunks + kLoTmemChunks;   // 32-column P blocks in tensor memory
constexpr int kThreads = 320;
constexpr int kPairChains = 64;                   // chains of a pair
constexpr int kHalf = 32;                         // chains per CTA
constexpr uint32_t kRowBytes = 128;               // one row of a K-chunk: 32 floats
constexpr uint32_t kLoOff = kHalf * kRowBytes;    // remainder rows follow the head rows
constexpr uint32_t kBChunk = 2 * kLoOff;          // 64 rows (32 head, 32 remainder) x 128 B
constexpr uint32_t kBBytes = kChunks * kBChunk;   // the position tile
constexpr uint32_t kAHalf = 128 * 128;            // 128 rows of P x 32 floats
constexpr uint32_t kABytes = (kChunks - kLoTmemChunks) * kAHalf;   // P remainder chunks 4-7
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColAcc = 0;                   // accumulators: 128 columns
constexpr uint32_t kColLoProduct = 32;            // the N = 64 product's column offset
constexpr uint32_t kColP = 128;                   // P block h (head chunk h, then remainder chunk h - 8) at kColP + 32 h
constexpr uint32_t kXferBytes = 4 * kHalf * kRowBytes;   // float32 positions of 32 chains x 128 dims
constexpr uint32_t kStateBytes = kPairChains * 128 * 4;   // current positions, this CTA's dims
// barriers (8), tmem slot, red [3][4][64], red_pair [3][64], peer_in [3][64],
// acc_flag [64], prob_s [64], DA state copy, flags, DA coefficients, pair
// sum, inverse temperatures [64], tempered log p after the decision [64],
// exchange flags [64], log u [64], current log p [64], |p0|^2 partials
// [2 transition parities][4 quarters][64]
constexpr uint32_t kSmall =
    8 * 8 + 16 + (3 * 4 * 64 + 3 * 64 + 3 * 64 + 64 + 64) * 4 + 128 + 16 + 32 + 16 + 5 * 64 * 4 +
    2 * 4 * 64 * 4;
constexpr size_t kSmemUsed = kBBytes + kABytes + 2 * kXferBytes + kStateBytes + kSmall + 1024;
// Above half of an SM's shared memory, so that one CTA runs per SM: a CTA
// allocates all 512 tensor-memory columns and must never queue in
// tcgen05.alloc behind another CTA of the launch.
constexpr size_t kSmem = kSmemUsed > 120 * 1024 ? kSmemUsed : 120 * 1024;
static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(kColP + 32 * kHalfChunks == kTmemCols, "tensor-memory columns");

struct PairArgs {
  StepArgs s;           // s.t / s.t_full: the first transition of the launch
  int* err;
  const float* Ptm;     // P chunks 0-6 in tensor-memory fill order (k_tmem_image)
  float* p0next;        // momenta of transition t in slot t % 2, per-thread blocks (scratch)
  int64_t p0_slot;      // floats per slot of p0next
  float* gb;            // cached gradients, per-thread blocks (scratch; not with the exchange step)
  float* wb;            // streaming: running mean, m2, batch sum, per-thread blocks (3 x p0_slot floats)
  int T;                // transitions in this launch
  long long keep_from;  // transition t_full >= keep_from writes output k = t_full - keep_from
  float* samples;       // [k][C x D] or null
  float* trace_eps;     // [k] or null
  uint8_t* trace_acc;   // [k][C] or null
  unsigned long long* stat;   // 3 statistic words (grid_barrier_sum), zero at launch
  float stat_hi_scale;  // 2^(f - 19), f the fraction bits of the fixed-point statistic
  double stat_scale;    // 2^-stat_frac / C
  uint8_t* swapped;     // exchange: [outer chains x (K - 1)] swap flags of the last transition
  int exchange;         // replica sets (K | 64): the exchange step after every transition
  unsigned long long grid_wait_ns;   // time after which the grid barrier gives up
  int unreachable_gen;  // > 0: this grid-barrier generation can never complete (tests)
  int samp_tma;         // the kept samples go out as tensor stores through the sample map
};

// Index of element e of float4 j of lane `lane` in the tensor-memory image:
// rank, 32-column P block h (0-7: head chunks 0-7, 8-11: remainder chunks
// 0-3), 16-column half q16, lane quarter q.  A warp's j-th float4 load of a
// 16-column block is 512 contiguous bytes.
__host__ __device__ constexpr int image_index(int rank, int h, int q16, int q, int j, int lane) {
  return ((((rank * kHalfChunks + h) * 2 + q16) * 4 + q) * 4 + j) * 128 + lane * 4;
}

__global__ void k_tmem_image(const float* __restrict__ Phi, const float* __restrict__ Plo, int D,
                             float* __restrict__ image) {
  constexpr int n = 2 * kHalfChunks * 2 * 4 * 4 * 32;   // float4 slots
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int r = v;
    const int lane = r % 32; r /= 32;
    const int j = r % 4; r /= 4;
    const int q = r % 4; r /= 4;
    const int q16 = r % 2; r /= 2;
    const int h = r % kHalfChunks;
    const int rank = r / kHalfChunks;
    const int row = rank * 128 + q * 32 + lane;
    const int col = (h < kChunks ? h : h - kChunks) * 32 + q16 * 16 + j * 4;
    const float* src = h < kChunks ? Phi : Plo;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < D && col < D)            // D % 4 == 0: all four in or out
      val = *reinterpret_cast<const float4*>(src + static_cast<int64_t>(row) * D + col);
    *reinterpret_cast<float4*>(image + image_index(rank, h, q16, q, j, lane)) = val;
  }
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// the leader's 64 deciding threads (epilogue warps 2 and 3)
__device__ __forceinline__ void deciders_barrier() { asm volatile("bar.sync 2, 64;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence_cta() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// v[c] summed over the warp's lanes, for all 32 c at once: 31 shuffles
// (each round halves the values a lane keeps); lane c ends with chain c's sum.
__device__ __forceinline__ float transpose_reduce32(float (&v)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const float send = upper ? v[k] : v[k + w];
      const float keep = upper ? v[k + w] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

// The momenta of slots 4 g .. 4 g + 3 of the epilogue thread of dim d (D % 4
// == 0) at transition tn: slot i < 16 is chain chain_peer + i, slot i >= 16
// chain chain_own + i - 16; slots past nv_peer / nv_own (chains >= C) are
// zero.  One Philox block (counter (d / 4, chain, tn)) holds a chain's
// momenta of dims 4 (d / 4) .. 4 (d / 4) + 3, the dims of the lane quad:
// lane m of the quad draws the block of slot 4 g + m's chain, and four
// rounds of shuffles hand each lane its own dim of all four blocks -- the
// same normals as one block per slot, for a quarter of the Philox rounds and
// half of the Box-Muller transforms.  Every lane of the warp takes part.
__device__ __forceinline__ void draw_quad(uint64_t seed, int d, int lane, uint32_t chain_peer, uint32_t chain_own,
                                          int nv_peer, int nv_own, int g, uint32_t tn, float (&v)[4]) {
  const int m = lane & 3;
  const int im = 4 * g + m;
  const uint32_t chain = im < 16 ? chain_peer + static_cast<uint32_t>(im) : chain_own + static_cast<uint32_t>(im - 16);
  const float4 n = momentum4(seed, static_cast<uint32_t>(d >> 2), chain, tn);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int snd = (m - k) & 3;      // component the reading lane m - k needs
    const float send = snd == 0 ? n.x : snd == 1 ? n.y : snd == 2 ? n.z : n.w;
    const int src = (m + k) & 3;      // slot 4 g + src's chain, drawn by quad lane src
    const float got = __shfl_sync(0xffffffffu, send, (lane & ~3) | src);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = src == e ? got : v[e];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int ie = 4 * g + e;
    v[e] = (ie < 16 ? ie < nv_peer : ie - 16 < nv_own) ? v[e] : 0.f;
  }
}

// The acceptance statistic of dual averaging (the mean acceptance
// probability over all chains) in fixed point: a chain's probability, a
// float32 in [0, 1], as a multiple of 2^-f, f = stat_frac_bits(C) (38 up to
// 8191 chains), so that the sum over C chains stays below 2^51.  Integer
// addition makes the sum independent of the order in which the CTAs add.
// One 64-bit word carries a generation's sum (bits 0-51) and its arrival
// count (bits 52-63), so the grid barrier and the reduction are one atomic
// per CTA.  (The statistic differs from a float64 sum by at most 2^-39 per
// chain at f = 38, far inside the tolerance the step sizes are checked to.)
constexpr unsigned long long kArriveOne = 1ull << 52;
constexpr unsigned long long kStatMask = kArriveOne - 1;

int stat_frac_bits(int64_t C) {
  int b = 0;
  while ((int64_t{1} << b) <= C) ++b;     // C < 2^b
  return b <= 13 ? 38 : std::max(20, 51 - b);
}

// round(p 2^frac) to nearest even, from two 32-bit conversions: with
// hi_scale = 2^(frac - 19), u = trunc(p hi_scale) and the fraction r of p
// hi_scale (both exact), the value is u 2^19 + rint(r 2^19).  (A conversion
// to 64 bits takes the float64 pipe, which is slow on this part.)
__device__ __forceinline__ unsigned long long prob_fixed(float p, float hi_scale) {
  const float v = p * hi_scale;
  const float u = truncf(v);
  return (static_cast<unsigned long long>(static_cast<unsigned>(u)) << 19) +
         __float2uint_rn((v - u) * 524288.0f);
}
// the mean from a sum word: scale = 2^-frac / C, formed on the host (one
// multiply here instead of a float64 division)
__device__ __forceinline__ double stat_mean(unsigned long long word, double scale) {
  return static_cast<double>(word & kStatMask) * scale;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* w, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(w), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* w) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
  return v;
}

// Grid barrier and statistic sum of a cooperative launch, generation `gen`
// (1, 2, ...) in word gen % 3 of `words` (all three zero at launch): adds
// this CTA's arrival and partial sum, waits until every CTA has arrived and
// returns the generation's word in *total.  The CTA whose arrival completes
// generation gen clears word (gen + 1) % 3, which generation gen - 1 used:
// every CTA has read it before arriving here, and generation gen + 2 adds
// to it only after every CTA (this one included, whose acq_rel arrival
// orders the clearing store first) has arrived at generation gen + 1.
// Bounded: false after `limit_ns`.  Generation `unreachable` (tests of the
// give-up path) waits for one arrival more than there are CTAs.  (Not
// inlined: inlined, it made the register allocator spill in the kernel.)
__device__ __noinline__ bool grid_barrier_sum(unsigned long long* words, unsigned gen, unsigned long long part,
                                                 unsigned long long limit_ns, int unreachable,
                                                 unsigned long long* total) {
  unsigned long long* w = words + gen % 3u;
  const unsigned long long target = gridDim.x + (static_cast<int>(gen) == unreachable ? 1u : 0u);
  unsigned long long cur = atom_add_acq_rel(w, kArriveOne + part) + kArriveOne + part;
  if ((cur >> 52) == target) {
    words[(gen + 1u) % 3u] = 0ull;
  } else {
    const unsigned long long t0 = ptx::global_timer_ns();
    while (((cur = ld_acquire_u64(w)) >> 52) < target) {
      if (ptx::global_timer_ns() - t0 > limit_ns) return false;
    }
  }
  *total = cur;
  return true;
}

// TEMPERED (replica exchange, Section 2.2): row r of the pair targets
// p^beta_r, beta_r = betas[(pair_base + r) % K].  Its gradient is
// -beta_r P x = -P (beta_r x), so the MMA operand tiles hold beta_r x and the
// epilogue, the energies and the cached log p / gradient come out tempered
// with no other change.  With fa.exchange (K divides 64, so a pair holds
// whole replica sets) the launch also takes the exchange step after every
// transition: the leader's deciding threads decide the adjacent pairs
// (k, k + 1), k = t mod 2, 2 + t mod 2, ..., through remc_swap_accept, and
// both CTAs swap the rows of their dims, rescaling the cached gradients,
// before the kept sample is written.
template <bool TEMPERED>
__global__ void __launch_bounds__(kThreads, 1)
k_gauss_pair(const __grid_constant__ CUtensorMap mPhi, const __grid_constant__ CUtensorMap mPlo,
             const __grid_constant__ CUtensorMap mSamp, PairArgs fa) {
  const StepArgs& a = fa.s;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* Bt = smem;                                      // positions: [8 K-chunks][head 32 rows, remainder 32 rows]
  uint8_t* As = Bt + kBBytes;                              // P remainder chunks 4-7
  uint8_t* Stg = As + kABytes;                             // outgoing float32 positions [4][32 rows][32 dims]
  uint8_t* Rcv = Stg + kXferBytes;                         // incoming float32 positions, same layout
  float* xs = reinterpret_cast<float*>(Rcv + kXferBytes);  // [64 chains][128 dims] current position
  uint64_t* a7_full = reinterpret_cast<uint64_t*>(xs + kPairChains * 128);
  uint64_t* acc_full = a7_full + 1;
  uint64_t* own_full = acc_full + 1;      // all epilogue threads: accumulators read, own K-chunks written
  uint64_t* in_full = own_full + 1;       // the other CTA's float32 positions have landed in Rcv
  uint64_t* fwd_own = in_full + 1;        // leader: the peer's own_full, forwarded
  uint64_t* fwd_in = fwd_own + 1;         // leader: the peer's split_full, forwarded
  uint64_t* sums_in = fwd_in + 1;         // the other CTA's partial sums have landed
  uint64_t* split_full = sums_in + 1;     // all epilogue threads: the received positions split into the tile
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(split_full + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);   // [3 sums][4 quarters][64 chains]
  float* red_pair = red + 3 * 4 * 64;                     // [3][64] this CTA's sums
  float* peer_in = red_pair + 3 * 64;                     // [3][64] the other CTA's sums
  int* acc_flag = reinterpret_cast<int*>(peer_in + 3 * 64);   // [64]
  float* prob_s = reinterpret_cast<float*>(acc_flag + 64);    // [64]
  DAState* da_s = reinterpret_cast<DAState*>(prob_s + 64);    // this CTA's copy (T > 1)
  int* abort_s = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(da_s) + 128);
  uint32_t* acc_mask_s = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(da_s) + 136);   // [2]
  DACoef* coef_s = reinterpret_cast<DACoef*>(reinterpret_cast<uint8_t*>(da_s) + 144);
  // the pair's fixed-point statistic, then the generation's word
  unsigned long long* psum_s = reinterpret_cast<unsigned long long*>(reinterpret_cast<uint8_t*>(da_s) + 176);
  float* beta_s = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(da_s) + 192);   // [64]
  float* lpn_s = beta_s + 64;                             // [64] exchange: log p after the decision
  int* swp_s = reinterpret_cast<int*>(lpn_s + 64);        // [64] exchange: row r and r + 1 swap
  float* lu_s = reinterpret_cast<float*>(swp_s + 64);     // [64] log u of this transition's accept test
  float* lpc_s = lu_s + 64;                               // [64] log p of the chains' current state
  float* kin_s = lpc_s + 64;                              // [2][4][64] |p0|^2 of transition t at t % 2

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_rank();              // 0: leader, 1: peer
  const int C = a.C, D = a.D, L = a.L, T = fa.T;
  const int nk = (D + 31) >> 5;
  const int nsm = nk > kLoTmemChunks ? nk - kLoTmemChunks : 0;   // P remainder chunks in shared memory
  const int pair_base = (blockIdx.x >> 1) * kPairChains;
  const bool persistent = T > 1;
  constexpr uint16_t kPairMask = 0x3;
  static_assert(sizeof(DAState) <= 128, "DA state copy");

  if (threadIdx.x == 0) {
    ptx::mbar_init(a7_full, 1);
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(own_full, 256);        // every epilogue thread
    ptx::mbar_init(in_full, 1);           // armed with the copy bytes by one epilogue thread
    ptx::mbar_init(split_full, 256);      // every epilogue thread
    ptx::mbar_init(fwd_own, 1);
    ptx::mbar_init(fwd_in, 1);
    ptx::mbar_init(sums_in, 1);            // armed each transition with the other CTA's 768 bytes
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mPhi);
    ptx::prefetch_tensormap(&mPlo);
    if (persistent) *da_s = *a.da;
    *abort_s = 0;
  }
  if (warp == 0) {
    ptx::tmem_alloc_pair(tmem_slot, kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  if (TEMPERED && threadIdx.x < kPairChains)
    beta_s[threadIdx.x] = a.betas[(pair_base + static_cast<int>(threadIdx.x)) % a.K];
  // position tile and staging start zeroed: dims >= D and chains >= C are never written
  for (uint32_t i = threadIdx.x; i < kBBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(Bt)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t i = threadIdx.x; i < kXferBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(Stg)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();      // both CTAs' barriers and tensor memory exist
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t peer = 1u - rank;
  bool ok = true;

  // epilogue-thread state (warps 2-9)
  const int ew = warp - 2;
  const int sub = ew >> 2;                // rows 16 sub .. 16 sub + 15 of each chain half
  const int quarter = warp & 3;           // tensor-memory lane quarter
  const int dl = quarter * 32 + lane;     // this CTA's dim index 0..127
  const int d = static_cast<int>(rank) * 128 + dl;
  const bool dvalid = warp >= 2 && d < D;
  float p[kHalf], x[kHalf];

  if (warp == 0) {
    if (lane == 0 && nsm > 0) {
      // ---- P remainder chunks 4-7 of this CTA's rows, once, completing on the leader's barrier
      if (rank == 0) ptx::mbar_arrive_expect_tx(a7_full, 2u * static_cast<uint32_t>(nsm) * kAHalf);
      const uint32_t bar = ptx::mapa(ptx::smem_u32(a7_full), 0);
      for (int c = 0; c < nsm; ++c)
        ptx::tma_load_2d_to_bar(As + c * kAHalf, &mPlo, bar, (kLoTmemChunks + c) * 32,
                                static_cast<int>(rank) * 128);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---- MMA issuer (leader): M = 256 across the pair
      constexpr uint32_t idesc_wide = ptx::idesc_tf32(256, 2 * kPairChains);   // head + remainder rows
      constexpr uint32_t idesc_head = ptx::idesc_tf32(256, kPairChains);       // head rows only
      if (nsm > 0 && !ptx::mbar_wait(a7_full, 0)) {
        atomicCAS(fa.err, 0, 1);
        ok = false;
      }
      // one K-chunk: 4 K-steps x 2 products (P_hi [x_hi; x_lo] with the head
      // from tensor memory, then P_lo x_hi with the remainder from tensor
      // memory for chunks 0-3 and from shared memory for chunks 4-7)
      auto chunk_mmas = [&](int kc, bool& first) {
        const uint32_t b = ptx::smem_u32(Bt + kc * kBChunk);
        if (kc < kLoTmemChunks) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t db = ptx::sw128_kmajor_desc(b + 32 * j);
            const uint32_t ahi = tmem + kColP + 32 * kc + 8 * j;
            const uint32_t alo = tmem + kColP + 32 * (kChunks + kc) + 8 * j;
            ptx::mma_tf32_pair_tmem_a(tmem + kColAcc, ahi, db, idesc_wide, first ? 0u : 1u);
            ptx::mma_tf32_pair_tmem_a(tmem + kColAcc + kColLoProduct, alo, db, idesc_head, 1u);
            first = false;
          }
        } else {
          const uint32_t alo = ptx::smem_u32(As + (kc - kLoTmemChunks) * kAHalf);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t db = ptx::sw128_kmajor_desc(b + 32 * j);
            const uint32_t ahi = tmem + kColP + 32 * kc + 8 * j;
            ptx::mma_tf32_pair_tmem_a(tmem + kColAcc, ahi, db, idesc_wide, first ? 0u : 1u);
            ptx::mma_tf32_pair(tmem + kColAcc + kColLoProduct, ptx::sw128_kmajor_desc(alo + 32 * j), db,
                               idesc_head, 1u);
            first = false;
          }
        }
      };
      // gradient step s (all transitions of the launch) consumes write s
      for (int s = 0; s < T * L && ok; ++s) {
        const uint32_t ph = s & 1;
        bool first = true;
        // K-chunks 4-7: leader half received from the peer and split here,
        // peer half local there; own_full and fwd_own also mean both CTAs'
        // epilogues have read the accumulators this step overwrites
        if (!ptx::mbar_wait(own_full, ph) || !ptx::mbar_wait(split_full, ph) ||
            !ptx::mbar_wait(fwd_own, ph)) {
          atomicCAS(fa.err, 0, 2);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int kc = 4; kc < nk; ++kc) chunk_mmas(kc, first);
        // K-chunks 0-3: leader half local, peer half received from the leader
        // and split there
        if (!ptx::mbar_wait(fwd_in, ph)) {
          atomicCAS(fa.err, 0, 3);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int kc = 0; kc < min(nk, 4); ++kc) chunk_mmas(kc, first);
        ptx::mma_commit_pair(acc_full, kPairMask);
      }
    } else if (lane == 0) {
      // ---- peer: forward both completions of this CTA's tile to the leader
      const uint32_t own_leader = ptx::mapa(ptx::smem_u32(fwd_own), 0);
      const uint32_t in_leader = ptx::mapa(ptx::smem_u32(fwd_in), 0);
      for (int s = 0; s < T * L; ++s) {
        const uint32_t ph = s & 1;
        if (!ptx::mbar_wait(own_full, ph)) {
          atomicCAS(fa.err, 0, 5);
          break;
        }
        ptx::mbar_arrive_remote(own_leader);
        if (!ptx::mbar_wait(split_full, ph)) {
          atomicCAS(fa.err, 0, 6);
          break;
        }
        ptx::mbar_arrive_remote(in_leader);
      }
    }
  } else {
    // ---- epilogue, both CTAs
    // Element i (0..31) of this thread is dim d of pair row rowi(i): the
    // first 16 are 16 of the peer's chains, whose float32 positions are
    // staged and pushed to the peer as soon as they are done; the last 16
    // are 16 of this CTA's own chains, split into head and remainder and
    // written straight into its tile.  Each step's copy thus starts after
    // half of the epilogue, and the other half overlaps it; the receiving
    // CTA splits the positions it gets into its own tile.  (Sending float32
    // instead of head and remainder halves the bytes crossing the pair:
    // 32 KB took about 0.9 us.)
    auto rowi = [&](int i) {
      return static_cast<int>(i < 16 ? peer : rank) * kHalf + sub * 16 + (i & 15);
    };
    // Tile addresses: head row r of K-chunk kc, column c, sits at
    // kc * kBChunk + (r / 8) * 1024 + sw[r % 8] + (c % 4) * 4 (the 128-byte
    // swizzle; sw depends on c / 4, and c = lane), its remainder kLoOff
    // further.
    const uint32_t own_hi0 = ptx::smem_u32(Bt) + static_cast<uint32_t>((d >> 5) * kBChunk + (d & 3) * 4);
    // the received positions of quarter q (the other CTA's dims) go to K-chunk 4 peer + q
    const uint32_t rcv_hi0 =
        ptx::smem_u32(Bt) + static_cast<uint32_t>((4 * static_cast<int>(peer) + quarter) * kBChunk + (lane & 3) * 4);
    // float32 transfer buffers: [quarter][row 0..31][lane], 128 B per row;
    // this thread's rows are 16 sub .. 16 sub + 15
    const uint32_t xfer_off = static_cast<uint32_t>(((quarter * kHalf + sub * 16) * 32 + lane) * 4);
    const uint32_t stg_a = ptx::smem_u32(Stg) + xfer_off;
    const uint32_t rcv_a = ptx::smem_u32(Rcv) + xfer_off;
    uint32_t sw[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) sw[r] = r * kRowBytes + (((((dl & 31) >> 2) ^ r) & 7) << 4);
    const int nv_peer = dvalid ? max(0, min(16, C - (pair_base + static_cast<int>(peer) * kHalf + sub * 16))) : 0;
    const int nv_own = dvalid ? max(0, min(16, C - (pair_base + static_cast<int>(rank) * kHalf + sub * 16))) : 0;
    auto valid = [&](int i) { return i < 16 ? i < nv_peer : i - 16 < nv_own; };
    auto xrow = [&](int i) -> float& { return xs[rowi(i) * 128 + dl]; };
    // element index of (pair row of element i, dim d) in the [C x D] arrays
    auto elem = [&](int i) { return static_cast<int64_t>(pair_base + rowi(i)) * D + d; };
    // The per-thread blocks of the scratch arrays fa.gb and fa.p0next: slot i
    // of the thread of dim d (d < D) is float i % 4 of float4
    // ((pair * 2 + sub) * 8 + i / 4) * D + d, so that a warp moves 512
    // contiguous bytes per float4 access (8 accesses for the 32 slots where
    // the [C x D] layout took 32).
    const int64_t blk4 = (static_cast<int64_t>(blockIdx.x >> 1) * 2 + sub) * 8 * D + d;
    // With the exchange step, rows swap: when the replica count divides 16
    // both rows of a swapped pair are this thread's (xblk) and the cached
    // gradients keep their per-thread blocks; otherwise they stay [C x D].
    const bool xchg = TEMPERED && fa.exchange;
    const bool xblk = xchg && a.K > 0 && 16 % a.K == 0;
    const bool gblocks = !xchg || xblk;
    // this thread's 32 slots from / to a per-thread block array
    auto blk_load = [&](const float* base, float (&v)[kHalf]) {
      const float4* b4 = reinterpret_cast<const float4*>(base) + blk4;
#pragma unroll
      for (int j = 0; j < kHalf / 4; ++j) {
        const float4 u = b4[static_cast<int64_t>(j) * D];
        v[4 * j] = u.x; v[4 * j + 1] = u.y; v[4 * j + 2] = u.z; v[4 * j + 3] = u.w;
      }
    };
    auto blk_store = [&](float* base, const float (&v)[kHalf]) {
      float4* b4 = reinterpret_cast<float4*>(base) + blk4;
#pragma unroll
      for (int j = 0; j < kHalf / 4; ++j)
        b4[static_cast<int64_t>(j) * D] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    };
    // Streaming driver: this thread's running moments (mean, m2 and, with
    // batches, the batch sum) stay in per-thread blocks during the launch,
    // read from the [C x D] arrays at its start and written back at its
    // end; a kept transition then takes 8 float4 loads and stores per array
    // where the [C x D] layout took 32 scalar ones.
    const bool wblocks = a.w.mean != nullptr && a.t_full + T > fa.keep_from && dvalid;
    const int n_wfields = a.w.bsize > 0 ? 3 : 2;
    auto wfield = [&](int k) { return reinterpret_cast<float4*>(fa.wb + k * fa.p0_slot) + blk4; };
    auto warray = [&](int k) { return k == 0 ? a.w.mean : k == 1 ? a.w.m2 : a.w.bsum; };
    auto wblk_sync = [&](bool in) {
      for (int k = 0; k < n_wfields; ++k) {
        float4* b4 = wfield(k);
        float* arr = warray(k);
#pragma unroll 1
        for (int g = 0; g < kHalf / 4; ++g) {
          if (in) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = valid(4 * g + e) ? arr[elem(4 * g + e)] : 0.f;
            b4[static_cast<int64_t>(g) * D] = make_float4(v[0], v[1], v[2], v[3]);
          } else {
            const float4 u = b4[static_cast<int64_t>(g) * D];
            const float v[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (valid(4 * g + e)) arr[elem(4 * g + e)] = v[e];
          }
        }
      }
    };
    // position of element i: the peer's chains as float32 into staging,
    // this CTA's own split into its tile
    auto store_x = [&](int i, float xi) {
      if (valid(i)) {
        if (TEMPERED) xi *= beta_s[rowi(i)];
        if (i < 16) {
          asm volatile("st.shared.f32 [%0], %1;" ::"r"(stg_a + i * kRowBytes), "f"(xi) : "memory");
        } else {
          float hi, lo;
          split_tf32(xi, hi, lo);
          const int r = sub * 16 + (i & 15);
          const uint32_t a0 = own_hi0 + (r >> 3) * 1024 + sw[r & 7];
          asm volatile("st.shared.f32 [%0], %1;" ::"r"(a0), "f"(hi) : "memory");
          asm volatile("st.shared.f32 [%0], %1;" ::"r"(a0 + kLoOff), "f"(lo) : "memory");
        }
      }
    };
    // Half h of the peer's half is written: the warp pushes its staged rows
    // 8 h .. 8 h + 7 (1 KB of float32 positions) to the peer's receive
    // buffer, completing on the peer's in_full.  (The transfer is bound by
    // the bandwidth between the two SMs: the first half starts it while the
    // second is computed.)
    auto publish_stage = [&](int h) {
      proxy_fence_cta();          // generic stores -> async proxy (bulk copy)
      __syncwarp();
      if (lane == 0) {
        const uint32_t off = static_cast<uint32_t>(quarter * kHalf + sub * 16 + 8 * h) * kRowBytes;
        ptx::bulk_copy_to_cluster(ptx::mapa(ptx::smem_u32(Rcv + off), peer), Stg + off, 8 * kRowBytes,
                                  ptx::mapa(ptx::smem_u32(in_full), peer));
      }
    };
    // The own half is written: every thread arrives on own_full once its
    // accumulator reads are done; one thread arms the incoming copy bytes.
    auto publish_own = [&]() {
      proxy_fence_cta();          // generic stores -> async proxy (MMA)
      ptx::tc_fence_before();     // this thread's accumulator reads precede the next MMA
      ptx::mbar_arrive_local(own_full);
      if (ew == 0 && lane == 0) ptx::mbar_arrive_expect_tx(in_full, kXferBytes);
    };
    // Write s of the tile (s = 0, 1, ...): once the other CTA's positions
    // have landed, this thread splits 16 of them (rows 16 sub .. 16 sub + 15
    // of this CTA's chains, dim 128 peer + 32 quarter + lane) into the tile,
    // eight at a time, and joins split_full.  Rows and dims with nothing to
    // send arrive as zeros.
    auto split_received = [&](int s) {
      if (!ptx::mbar_wait(in_full, s & 1)) {
        atomicCAS(fa.err, 0, 10);
        ok = false;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v[k]) : "r"(rcv_a + (8 * h + k) * kRowBytes) : "memory");
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          float hi, lo;
          split_tf32(v[k], hi, lo);
          const int r = sub * 16 + 8 * h + k;
          const uint32_t a0 = rcv_hi0 + (r >> 3) * 1024 + sw[k];
          asm volatile("st.shared.f32 [%0], %1;" ::"r"(a0), "f"(hi) : "memory");
          asm volatile("st.shared.f32 [%0], %1;" ::"r"(a0 + kLoOff), "f"(lo) : "memory");
        }
      }
      proxy_fence_cta();
      ptx::mbar_arrive_local(split_full);
    };
    // The gradient of elements 16 cb .. 16 cb + 15 is minus the sum of their
    // two accumulator columns: (CTA q, row r) -> column 64 q + r and 64 q + r + 32.
    const uint32_t acc_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + kColAcc;
    auto load_acc = [&](int cb, float (&acc)[16]) {
      const uint32_t col = acc_base + static_cast<uint32_t>(static_cast<int>(cb == 0 ? peer : rank) * 64 + sub * 16);
      ptx::tmem_ld8x2_sum(col, col + 32, acc);
      ptx::tmem_ld8x2_sum(col + 8, col + 40, acc + 8);
    };
    auto wait_acc = [&](int s) {
      if (!ptx::mbar_wait(acc_full, s & 1)) {
        atomicCAS(fa.err, 0, 4);
        ok = false;
      }
      ptx::tc_fence_after();
    };
    auto chain_of = [&](int i) { return static_cast<uint32_t>(pair_base + rowi(i)) + a.chain_offset; };
    constexpr int kGroups = kHalf / 4;
    // The next transition's momenta, parked in the per-thread blocks: 64
    // items (epilogue warp w, slot group g) per transition, each one float4
    // per lane of w's block.  The six epilogue warps off the MMA issuer's
    // sub-partition (warp % 4 != 1) draw them all, item k + 6 n for the k-th
    // of them, n items per gradient wait: drawing in warps 5 and 9 measured
    // 0.1 us per step more MMA issue time.  Transition tn's momenta go to
    // slot tn % 2, so that no warp overwrites momenta another has yet to load.
    const bool drawer = (warp & 3) != 1;
    const int dk = warp < 5 ? warp - 2 : warp - 3;           // 0..5 for the drawers
    const int n_items = drawer ? (8 * kGroups - dk + 5) / 6 : 0;
    const int per_wait = (8 * kGroups / 6 + 1 + L - 1) / L;   // items of a drawer per wait (at most 11)
    auto draw_next = [&](int n0, int n1, uint32_t tn) {
      for (int n = n0; n < min(n1, n_items); ++n) {
        const int item = dk + 6 * n;
        const int tw = 2 + (item >> 3), g = item & 7;          // warp whose slots, slot group
        const int tq = tw & 3, tsub = (tw - 2) >> 2;
        if (static_cast<int>(rank) * 128 + tq * 32 >= D) {   // warp-uniform: no dims, no momenta,
          if (lane < 4) {                                     // and zero |p0|^2 partials
            const int i = 4 * g + lane;
            const int row = (i < 16 ? static_cast<int>(peer) : static_cast<int>(rank)) * kHalf + tsub * 16 + (i & 15);
            kin_s[((tn & 1u) * 4 + static_cast<uint32_t>(tq)) * 64 + row] = 0.f;
          }
          continue;
        }
        const int dt = static_cast<int>(rank) * 128 + tq * 32 + lane;
        const bool dv = dt < D;
        const int rp = pair_base + static_cast<int>(peer) * kHalf + tsub * 16;
        const int ro = pair_base + static_cast<int>(rank) * kHalf + tsub * 16;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        draw_quad(a.seed, dt, lane, static_cast<uint32_t>(rp) + a.chain_offset,
                  static_cast<uint32_t>(ro) + a.chain_offset, dv ? max(0, min(16, C - rp)) : 0,
                  dv ? max(0, min(16, C - ro)) : 0, g, tn, v);
        if (dv) {
          const int64_t b4 = (static_cast<int64_t>(blockIdx.x >> 1) * 2 + tsub) * 8 * D + dt;
          reinterpret_cast<float4*>(fa.p0next + (tn & 1u) * fa.p0_slot)[b4 + static_cast<int64_t>(g) * D] =
              make_float4(v[0], v[1], v[2], v[3]);
        }
        // the four chains' |p0|^2 over warp tw's 32 dims, for transition tn's
        // decision: the xor butterfly pairs the lanes as the transpose
        // reduction at the top of a transition does, so the sums agree bit
        // for bit (each step adds two partial sums, and a + b == b + a)
        float w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = dv ? v[e] * v[e] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int e = 0; e < 4; ++e) w[e] += __shfl_xor_sync(0xffffffffu, w[e], o);
        if (lane == 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = 4 * g + e;
            const int row = (i < 16 ? static_cast<int>(peer) : static_cast<int>(rank)) * kHalf + tsub * 16 + (i & 15);
            kin_s[((tn & 1u) * 4 + static_cast<uint32_t>(tq)) * 64 + row] = w[e];
          }
        }
      }
    };

    // P rows of this CTA (row = output dim d = TMEM lane) into tensor memory
    // from the pre-arranged image (coalesced): the two warps of a lane
    // quarter split the twelve 32-column blocks (head chunks 0-7, remainder
    // chunks 0-3) six and six
    {
      constexpr int kSplit = kHalfChunks / 2;
      for (int h = sub == 0 ? 0 : kSplit; h < (sub == 0 ? kSplit : kHalfChunks); ++h) {
        if ((h < kChunks ? h : h - kChunks) >= nk) continue;
#pragma unroll
        for (int q16 = 0; q16 < 2; ++q16) {
          float v[16];
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const float4 u = *reinterpret_cast<const float4*>(
                fa.Ptm + image_index(static_cast<int>(rank), h, q16, quarter, q4, lane));
            v[4 * q4] = u.x; v[4 * q4 + 1] = u.y; v[4 * q4 + 2] = u.z; v[4 * q4 + 3] = u.w;
          }
          ptx::tmem_st16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + kColP + 32 * h + 16 * q16, v);
        }
      }
      ptx::tmem_wait_st();
    }
    // the chains' current positions, this CTA's dims (their gradients stay
    // in a.g, which the accepted proposals overwrite)
#pragma unroll 4
    for (int i = 0; i < kHalf; ++i) xrow(i) = valid(i) ? a.x[elem(i)] : 0.f;
    if (wblocks) wblk_sync(true);
    // At the top of every transition p holds the cached gradients g0 and x
    // the transition's momenta p0 (for the first one drawn here, for the
    // others loaded during the previous transition's accept step).
#pragma unroll
    for (int i = 0; i < kHalf; ++i) p[i] = valid(i) ? a.g[elem(i)] : 0.f;
    // the launch's cached gradients in this thread's block (the accept steps
    // keep them there; the last one writes them back to a.g)
    if (gblocks && dvalid) blk_store(fa.gb, p);
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      draw_quad(a.seed, d, lane, chain_of(0), chain_of(16), nv_peer, nv_own, g, a.t, v);
#pragma unroll
      for (int e = 0; e < 4; ++e) x[4 * g + e] = v[e];
    }
    // the deciding threads (warps 2-3 of both CTAs, chain pair_base + c):
    // the current log p of their chain, kept in shared memory from here on
    const int c = ew * 32 + lane;                 // 0..255; chains 0..63 decide
    if (c < kPairChains) lpc_s[c] = pair_base + c < C ? a.lp[pair_base + c] : 0.f;

    int nbar = 0;                           // grid barriers met so far (T > 1)
    int err_seen = 0;                       // warp 2 lane 0: the error flag at the last boundary
    for (int j = 0; j < T; ++j) {
      const uint32_t t = a.t + static_cast<uint32_t>(j);
      const bool more = j + 1 < T;
      const float eps = persistent ? da_s->eps : a.da->eps;
      // |p0|^2 partials of this warp's dims, one per chain: for the launch's
      // first transition here; later ones were summed by the warps that drew
      // the momenta
      if (j == 0) {
        float v[kHalf];
#pragma unroll
        for (int i = 0; i < kHalf; ++i) v[i] = x[i] * x[i];
        kin_s[((t & 1u) * 4 + static_cast<uint32_t>(quarter)) * 64 + rowi(lane)] = transpose_reduce32(v, lane);
      }
      // begin: p = p0 + eps/2 g0, x1 = x0 + eps p (the peer's half first);
      // every position is loaded before the first tile store, whose memory
      // clobber would otherwise serialise the loads
#pragma unroll
      for (int i = 0; i < kHalf; ++i) p[i] = fmaf(0.5f * eps, p[i], x[i]);
#pragma unroll
      for (int i = 0; i < kHalf; ++i) x[i] = xrow(i);
#pragma unroll
      for (int i = 0; i < kHalf; ++i) {
        x[i] = fmaf(eps, p[i], x[i]);
        store_x(i, x[i]);
        if (i == 7 || i == 15) publish_stage(i >> 3);
      }
      publish_own();
      split_received(j * L);
      // the accept test's log u, off the critical path
      if (c < kPairChains && pair_base + c < C)
        lu_s[c] = accept_log_uniform(a.seed, static_cast<uint32_t>(pair_base + c) + a.chain_offset, t);
      const int s0 = j * L;                 // gradient steps of this transition: s0 .. s0 + L - 1
      // steps 1 .. L-1: merged kick + drift
      for (int l = 1; l < L; ++l) {
        if (more) draw_next((l - 1) * per_wait, l * per_wait, t + 1);
        wait_acc(s0 + l - 1);
#pragma unroll
        for (int cb = 0; cb < kHalf / 16; ++cb) {
          float accv[16];
          load_acc(cb, accv);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int i = cb * 16 + k;
            p[i] = fmaf(-eps, accv[k], p[i]);
            x[i] = fmaf(eps, p[i], x[i]);
            store_x(i, x[i]);
            if (cb == 0 && (k == 7 || k == 15)) publish_stage(k >> 3);
          }
        }
        publish_own();
        split_received(s0 + l);
      }
      // step L: final half kick; <x, g> and |p|^2 partials
      if (more) draw_next((L - 1) * per_wait, n_items, t + 1);
      wait_acc(s0 + L - 1);
      {
        float v[kHalf];
#pragma unroll
        for (int cb = 0; cb < kHalf / 16; ++cb) {
          float accv[16];
          load_acc(cb, accv);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int i = cb * 16 + k;
            p[i] = fmaf(-0.5f * eps, accv[k], p[i]);
            v[i] = valid(i) ? -x[i] * accv[k] : 0.f;
          }
        }
        red[(0 * 4 + quarter) * 64 + rowi(lane)] = transpose_reduce32(v, lane);
#pragma unroll
        for (int i = 0; i < kHalf; ++i) v[i] = valid(i) ? p[i] * p[i] : 0.f;
        red[(1 * 4 + quarter) * 64 + rowi(lane)] = transpose_reduce32(v, lane);
      }
      // The momenta are spent: p takes the cached gradients (8 float4 loads
      // from this thread's block, in flight while the chains are decided; the
      // accepted ones are replaced below).  32 scalar loads of the [C x D]
      // cache here measured 1 us of issue time per transition.
      if (gblocks && dvalid) blk_load(fa.gb, p);
      // The error flag: the value read at the previous boundary raises the
      // abort flag, which every epilogue thread reads after the barrier below
      // (and acts on at the end of this transition), and this boundary's read
      // stays in flight: no barrier of its own.
      if (persistent && warp == 2 && lane == 0) {
        if (err_seen != 0) *abort_s = 1;
        err_seen = *reinterpret_cast<volatile int*>(fa.err);
      }
      epi_barrier();
      const bool stop = persistent && *reinterpret_cast<volatile int*>(abort_s) != 0;
      // Only the epilogue warps run this loop, so the two CTAs meet on an
      // mbarrier: each sends its partial sums to the other by asynchronous
      // stores that complete on the other's sums_in, and both decide every
      // chain of the pair from the same two partials (a + b equals b + a in
      // float32, so the decisions agree bit for bit); the leader writes the
      // kernel results.
      if (c < kPairChains) {
        const uint32_t bar = ptx::mapa(ptx::smem_u32(sums_in), peer);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          float sum = 0.f;
          const float* part = v < 2 ? red + v * 4 * 64 : kin_s + (t & 1u) * 4 * 64;
          for (int q = 0; q < 4; ++q) sum += part[q * 64 + c];
          red_pair[v * 64 + c] = sum;
          ptx::st_async_f32(ptx::mapa(ptx::smem_u32(&peer_in[v * 64 + c]), peer), sum, bar);
        }
      }
      const long long t_full = a.t_full + j;
      const long long k_out = t_full - fa.keep_from;
      if (c < kPairChains) {
        if (c == 0) ptx::mbar_arrive_expect_tx(sums_in, 3 * kPairChains * 4);
        if (!ptx::mbar_wait(sums_in, j & 1)) {
          atomicCAS(fa.err, 0, 8);
          ok = false;
        }
        const bool lead = rank == 0;
        // H_L and the Metropolis-Hastings decision, chain c of the pair
        const int chain = pair_base + c;
        float prob = 0.f;
        int acc = 0;
        if (chain < C) {
          const float xg = red_pair[c] + peer_in[c];
          const float pp = red_pair[64 + c] + peer_in[64 + c];
          const float kin0 = 0.5f * (red_pair[128 + c] + peer_in[128 + c]);
          const float lp0 = lpc_s[c];
          const float lp1 = 0.5f * xg;
          float la = (-lp0 + kin0) - (-lp1 + 0.5f * pp);
          if (!isfinite(la)) la = -INFINITY;
          acc = lu_s[c] < la;
          prob = accept_prob(la);
          if (TEMPERED && fa.exchange) {
            lpn_s[c] = acc ? lp1 : lp0;
          } else if (acc) {
            lpc_s[c] = lp1;
          }
          // log u is spent: its slot keeps log alpha for the kernel results,
          // written after the accept step (a proxy fence there would
          // otherwise wait for these global stores)
          lu_s[c] = la;
        }
        acc_flag[c] = acc;
        prob_s[c] = prob;
        // the decisions of rows 32 ew .. 32 ew + 31 as one word
        const unsigned accw = __ballot_sync(0xffffffffu, acc != 0);
        if (lane == 0) acc_mask_s[ew] = accw;
        if (TEMPERED && fa.exchange) {
          // the exchange step: row c decides the pair (c, c + 1) when it is
          // the lower replica of an active pair, then every row takes its
          // log p (swapped and rescaled where its pair swapped)
          deciders_barrier();
          const int Kr = a.K;
          const int row = pair_base + c;
          const int k = row % Kr;
          const uint32_t cout = static_cast<uint32_t>(row / Kr);
          int sw = 0;
          if (row < C && k < Kr - 1) {
            if ((k & 1) == static_cast<int>(t & 1u)) {
              float raw0, raw1;
              sw = remc_swap_accept(lpn_s[c], lpn_s[c + 1], beta_s[c], beta_s[c + 1], a.seed,
                                    static_cast<uint32_t>(k), cout, t, &raw0, &raw1);
            }
            if (ok && lead) fa.swapped[static_cast<int64_t>(cout) * (Kr - 1) + k] = static_cast<uint8_t>(sw);
          }
          swp_s[c] = sw;
          deciders_barrier();
          if (row < C) {
            float lpf = lpn_s[c];
            if (swp_s[c]) {                        // lower row of a swapped pair
              lpf = beta_s[c] * (lpn_s[c + 1] / beta_s[c + 1]);
            } else if (k > 0 && swp_s[c - 1]) {    // upper row of a swapped pair
              lpf = beta_s[c] * (lpn_s[c - 1] / beta_s[c - 1]);
            }
            lpc_s[c] = lpf;
            if (ok && lead) a.lp[row] = lpf;
          }
        }
        if (lead && blockIdx.x == 0 && c == 0 && k_out >= 0 && fa.trace_eps && ok) fa.trace_eps[k_out] = eps;
      }
      // the previous kept sample's bulk stores have read the positions
      // (warp 2 issues them) before anything below writes them
      if (warp == 2) ptx::bulk_wait_read();
      // decisions visible to every epilogue thread
      epi_barrier();
      // the accepted state (gradient from the accumulators) and the kept sample
      float* samp = (k_out >= 0 && fa.samples) ? fa.samples + k_out * static_cast<int64_t>(C) * D : nullptr;
      // streaming driver: running moments of the kept states instead of a trace
      const bool moments = k_out >= 0 && a.w.mean != nullptr;
      // The decisions of this thread's 32 rows first, then only global
      // accesses: shared-memory loads between the (possibly aliasing) global
      // stores would each wait for the previous one.  The accepted positions
      // go first, and (when a sample is kept) the proxy fence that hands them
      // to the trace's tensor store comes before the gradient accesses: a
      // fence waits for this thread's global accesses in flight.  An accepted
      // chain's gradient comes from the accumulators (and is stored as the
      // new cached gradient), a rejected chain's is loaded from the cache.
      // bit i: element i's chain was accepted (rows 16 sub .. 16 sub + 15 of
      // the peer's half, then of this CTA's)
      const uint32_t accm = ((acc_mask_s[peer] >> (16 * sub)) & 0xffffu) |
                            (((acc_mask_s[rank] >> (16 * sub)) & 0xffffu) << 16);
#pragma unroll
      for (int i = 0; i < kHalf; ++i)
        if (ok && valid(i) && ((accm >> i) & 1u)) xrow(i) = x[i];
      if (samp && !(TEMPERED && fa.exchange)) proxy_fence_cta();
#pragma unroll
      for (int cb = 0; cb < kHalf / 16; ++cb) {
        float accv[16];
        load_acc(cb, accv);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int i = cb * 16 + k;
          if (ok && valid(i) && ((accm >> i) & 1u)) {
            if (xchg && !xblk) a.g[elem(i)] = -accv[k];
            p[i] = -accv[k];
          }
        }
      }
      // the exchange step's row swaps when both rows are this thread's: the
      // positions in the shared rows, the cached gradients in p, rescaled as
      // the exchange kernel does (swapped pairs are disjoint: a row swapped
      // as the upper one is never the lower one of another)
      if (xblk) {
#pragma unroll
        for (int i = 0; i < kHalf - 1; ++i) {
          if ((i & 15) == 15) continue;
          const int r = rowi(i);
          if (ok && valid(i) && swp_s[r]) {
            float* x0 = &xs[r * 128 + dl];
            const float xa = x0[0], xb = x0[128];
            const float b0 = beta_s[r], b1 = beta_s[r + 1];
            x0[0] = xb;
            x0[128] = xa;
            const float ga = p[i], gb = p[i + 1];
            p[i] = gb / b1 * b0;
            p[i + 1] = ga / b0 * b1;
          }
        }
      }
      // the cached gradients: back to this thread's block, or, after the
      // launch's last transition, to a.g (with the exchange step and a
      // replica count not dividing 16, a.g is the cache throughout, and the
      // exchange below reloads p)
      if (gblocks && ok) {
        if (more) {
          if (dvalid) blk_store(fa.gb, p);
        } else {
#pragma unroll
          for (int i = 0; i < kHalf; ++i)
            if (valid(i)) a.g[elem(i)] = p[i];
        }
      }
      // the kernel results of chain c of the pair (the leader's deciders)
      if (rank == 0 && c < kPairChains && pair_base + c < C && ok) {
        const int chain = pair_base + c;
        const int acc = acc_flag[c];
        if (!(TEMPERED && fa.exchange) && acc) a.lp[chain] = lpc_s[c];
        a.is_accepted[chain] = static_cast<uint8_t>(acc);
        a.log_accept[chain] = lu_s[c];
        if (k_out >= 0 && fa.trace_acc) fa.trace_acc[k_out * C + chain] = static_cast<uint8_t>(acc);
      }
      if (xchg && !xblk) {
        // swap the state rows of this CTA's dims: the owner of the lower row
        // of each swapped pair exchanges both rows (gradients rescaled as the
        // exchange kernel does), then the kept sample is written
        epi_barrier();
#pragma unroll
        for (int i = 0; i < kHalf; ++i) {
          const int r = rowi(i);
          if (ok && valid(i) && swp_s[r]) {
            float* x0 = &xs[r * 128 + dl];
            float* g0 = a.g + elem(i);
            const float xa = x0[0], xb = x0[128];
            const float ga = g0[0], gb = g0[D];
            const float b0 = beta_s[r], b1 = beta_s[r + 1];
            x0[0] = xb;
            x0[128] = xa;
            g0[0] = gb / b1 * b0;
            g0[D] = ga / b0 * b1;
          }
        }
        // swapped rows took new cached gradients (the other row of a pair
        // may belong to another thread of this dim)
        epi_barrier();
        if (more) {
#pragma unroll
          for (int i = 0; i < kHalf; ++i) p[i] = valid(i) ? a.g[elem(i)] : 0.f;
        }
      }
      // The kept sample: this CTA's positions (64 rows of its dims) are
      // complete in shared memory, and one thread writes them to the trace as
      // one tensor store of the [64 chains x 128 dims] box (rows >= C and dims
      // >= D fall outside the tensor and are not written), waited for before
      // the next transition writes the rows.  (One bulk copy per chain row,
      // issued by the lanes of one warp, measured 2.1 us per transition.)
      if (samp) {
        if (TEMPERED && fa.exchange) proxy_fence_cta();    // the swapped rows
        epi_barrier();
        const int ndim = min(128, D - static_cast<int>(rank) * 128);
        if (fa.samp_tma) {
          if (warp == 2 && lane == 0 && ok && ndim > 0) {
            ptx::tma_store_3d(&mSamp, ptx::smem_u32(xs), static_cast<int>(rank) * 128, pair_base,
                              static_cast<int>(k_out));
            ptx::bulk_commit();
          }
        } else if (ok && ndim > 0) {
          // no sample map (a trace pointer without 16-byte alignment):
          // coalesced plain stores
          for (int e = ew * 32 + lane; e < kPairChains * ndim; e += 256) {
            const int r = e / ndim, cidx = e - r * ndim;
            if (pair_base + r < C)
              samp[static_cast<int64_t>(pair_base + r) * D + static_cast<int>(rank) * 128 + cidx] = xs[r * 128 + cidx];
          }
        }
      }
      // the next transition's momenta (drawn during this one's steps), loaded
      // once the positions are spent and after the proxy fence above (a fence
      // waits for the loads in flight)
      if (more) {
        asm volatile("" ::: "memory");
        if (dvalid) {
          blk_load(fa.p0next + ((t + 1u) & 1u) * fa.p0_slot, x);
        } else {
#pragma unroll
          for (int i = 0; i < kHalf; ++i) x[i] = 0.f;
        }
      }
      if (moments && ok && dvalid) {
        // (the coefficients take 64-bit divisions: only when moments are kept)
        const WelfordCoef wq = welford_coef(k_out, a.w.bsize);
        const bool batches = a.w.bsize > 0;
        float4* mb = wfield(0);
        float4* sb = wfield(1);
        float4* bb = wfield(2);
        // Welford's update (as welford_update) per slot, four slots a float4;
        // the batch means of a closing batch stay [C x D]
#pragma unroll 1
        for (int g = 0; g < kHalf / 4; ++g) {
          const int64_t o = static_cast<int64_t>(g) * D;
          const float4 m4 = mb[o], s4 = sb[o];
          const float4 c4 = batches ? bb[o] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float m0[4] = {m4.x, m4.y, m4.z, m4.w}, s0[4] = {s4.x, s4.y, s4.z, s4.w};
          const float b0[4] = {c4.x, c4.y, c4.z, c4.w};
          float m1[4], s1[4], b1[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = 4 * g + e;
            const float xv = xrow(i);
            if (k_out == 0) {
              m1[e] = xv;
              s1[e] = 0.f;
            } else {
              const float delta = xv - m0[e];
              m1[e] = fmaf(delta, wq.inv, m0[e]);
              s1[e] = fmaf(delta, xv - m1[e], s0[e]);
            }
            b1[e] = wq.pos == 0 ? xv : b0[e] + xv;
            if (batches && wq.closes && valid(i)) {
              const float bm = b1[e] * wq.inv_b;
              const int64_t ei = elem(i);
              if (wq.batch == 0) {
                a.w.bmean[ei] = bm;
                a.w.bm2[ei] = 0.f;
              } else {
                const float bm0 = a.w.bmean[ei], bs0 = a.w.bm2[ei];
                const float delta = bm - bm0;
                const float bn = fmaf(delta, wq.inv_j, bm0);
                a.w.bmean[ei] = bn;
                a.w.bm2[ei] = fmaf(delta, bm - bn, bs0);
              }
            }
          }
          mb[o] = make_float4(m1[0], m1[1], m1[2], m1[3]);
          sb[o] = make_float4(s1[0], s1[1], s1[2], s1[3]);
          if (batches) bb[o] = make_float4(b1[0], b1[1], b1[2], b1[3]);
        }
      }
      // dual averaging over all chains of the posterior
      if (persistent) {
        // Transitions that adapt (and the launch's last, whose statistic the
        // state reports) meet at the grid barrier, which also sums the
        // fixed-point statistic (the pair's sum from the leader, zero from
        // the peer; warp 2, lane 0), while warp 3 forms the update's
        // coefficients.  Every CTA then applies the same update to its own
        // copy of the state, as the one-transition launch does to the
        // context's.  The others only check the error flag: a step size
        // that does not adapt needs no statistic.
        const bool adapts = da_s->adapt && t_full < da_s->num_adapt;
        if (adapts || !more) {
          ++nbar;
          if (warp == 2) {
            unsigned long long v = rank == 0 ? prob_fixed(prob_s[lane], fa.stat_hi_scale) +
                                                   prob_fixed(prob_s[lane + 32], fa.stat_hi_scale)
                                             : 0ull;
            v = warp_sum_u64(v);
            if (lane == 0) {
              unsigned long long total = 0ull;
              if (!grid_barrier_sum(fa.stat, static_cast<unsigned>(nbar), v, fa.grid_wait_ns, fa.unreachable_gen,
                                    &total)) {
                atomicCAS(fa.err, 0, 7);
                *abort_s = 1;
              } else if (err_seen == 0) {
                // (warp 3's coefficients are ready after the barrier below)
                *psum_s = total;
              } else {
                *abort_s = 1;
              }
            }
          } else if (warp == 3 && lane == 0) {
            *coef_s = da_prepare(da_s, t_full);
          }
          epi_barrier();
          if (warp == 2 && lane == 0 && *reinterpret_cast<volatile int*>(abort_s) == 0)
            da_apply(da_s, *coef_s, stat_mean(*psum_s, fa.stat_scale), t_full);
          epi_barrier();
          if (*reinterpret_cast<volatile int*>(abort_s)) break;
        } else if (stop) {
          break;
        }
      } else if (warp == 2) {
        // one transition: the pair's sum for the last-CTA update below
        unsigned long long v =
            rank == 0 ? prob_fixed(prob_s[lane], fa.stat_hi_scale) + prob_fixed(prob_s[lane + 32], fa.stat_hi_scale)
                      : 0ull;
        v = warp_sum_u64(v);
        if (lane == 0) *psum_s = v;
      }
    }
    // the chains' final positions back to global memory (the gradients are there)
#pragma unroll 4
    for (int i = 0; i < kHalf; ++i)
      if (ok && valid(i)) a.x[elem(i)] = xrow(i);
    if (wblocks && ok) wblk_sync(false);
    if (persistent && blockIdx.x == 0 && threadIdx.x == 64 && !*abort_s) *a.da = *da_s;
    if (warp == 2) ptx::bulk_wait_all();      // the kept samples' bulk stores are done
  }
  // every copy into this CTA's tile has landed (immediate unless a wait gave up)
  if (warp == 1 && lane == 0) ptx::mbar_wait(in_full, (T * L - 1) & 1);
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, kTmemCols);
  }
  ptx::cluster_sync();
  if (!persistent && threadIdx.x == 64) {
    // One transition: every CTA adds its statistic to word 0 and its arrival
    // to word 1 (acq_rel: the sum is in place before the arrival counts); the
    // CTA that arrives last applies the dual-averaging update with the same
    // arithmetic as the multi-transition launch.  (The grid need not be
    // resident at once, so the sum and the count are separate words here.)
    atomicAdd(fa.stat, *psum_s);
    if (atom_add_acq_rel(fa.stat + 1, 1ull) + 1ull == gridDim.x)
      da_update(a.da, stat_mean(ld_acquire_u64(fa.stat), fa.stat_scale), a.t_full);
  }
}

}  // namespace

// Test support: the grid barrier's wait limit and an unreachable generation
// (set by hmc_debug_set_grid_barrier; read at every launch).
std::atomic<unsigned long long> g_grid_wait_ns{ptx::kWaitLimitNs};
std::atomic<int> g_unreachable_gen{0};

void set_grid_barrier_debug(unsigned long long wait_ns, int unreachable_gen) {
  g_grid_wait_ns.store(wait_ns);
  g_unreachable_gen.store(unreachable_gen);
}

unsigned gauss_pair_grid(int64_t C) {
  return static_cast<unsigned>(2 * ((C + kPairChains - 1) / kPairChains));
}

cudaError_t launch_gauss_pair_image(const float* Phi, const float* Plo, int D, float* image,
                                    cudaStream_t s) {
  static_assert(kGaussPairImageFloats == 2 * kHalfChunks * 2 * 4 * 4 * 32 * 4, "image size");
  k_tmem_image<<<static_cast<unsigned>(kGaussPairImageFloats / 4 / 256), 256, 0, s>>>(Phi, Plo, D, image);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gauss_pair_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_gauss_pair<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gauss_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kSmem));
}

// Whether all CTA pairs of a launch for C chains can be resident at once
// (the condition for a cooperative launch of several transitions).
bool gauss_pair_persistent_ok(int64_t C) {
  static int max_clusters = -1;
  if (max_clusters < 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (gauss_pair_setup() != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&n, k_gauss_pair<false>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    max_clusters = n;
  }
  return static_cast<int64_t>(gauss_pair_grid(C) / 2) <= max_clusters;
}

// T transitions starting at a.t / a.t_full.  T > 1 needs a cooperative
// launch; the statistic words (tc.pair_stat) are zeroed here.
cudaError_t launch_gauss_pair_transitions(const StepArgs& a, GaussTc& tc, int T, long long keep_from,
                                          float* samples, float* trace_eps, uint8_t* trace_acc,
                                          cudaStream_t s, KernelTimer* timer, uint8_t* swapped) {
  if (swapped && (!a.betas || a.K < 2 || kPairChains % a.K != 0)) return cudaErrorInvalidValue;
  // the kept samples of this launch, outputs 0 .. t_full + T - 1 - keep_from,
  // as one [64 chains x 128 dims] tensor store per CTA and transition
  CUtensorMap mSamp{};
  const long long nkeep = a.t_full + T - keep_from;
  const bool samp_tma = samples && nkeep > 0 && make_sample_map(&mSamp, samples, a.D, a.C, nkeep);
  PairArgs fa{a, tc.err, tc.Ptm, tc.pair_p, gauss_pair_padded_chains(a.C) * a.D, tc.pair_g, tc.pair_w,
              T, keep_from, samples, trace_eps, trace_acc, tc.pair_stat,
              std::ldexp(1.0f, stat_frac_bits(a.C) - 19),
              std::ldexp(1.0, -stat_frac_bits(a.C)) / static_cast<double>(a.C),
              swapped, swapped ? 1 : 0, g_grid_wait_ns.load(), g_unreachable_gen.load(), samp_tma ? 1 : 0};
  {
    cudaError_t e = cudaMemsetAsync(tc.pair_stat, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gauss_pair_grid(a.C));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = T > 1 ? 2 : 1;
  if (timer) timer->begin(s);
  cudaError_t e = a.betas ? cudaLaunchKernelEx(&cfg, k_gauss_pair<true>, tc.mPhi128, tc.mPlo128, mSamp, fa)
                          : cudaLaunchKernelEx(&cfg, k_gauss_pair<false>, tc.mPhi128, tc.mPlo128, mSamp, fa);
  if (timer) timer->end(s);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_gauss_pair_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                         KernelTimer* timer) {
  // one transition: its outputs, if any, are output 0
  const bool keep = a.sample_out || a.trace_eps || a.trace_acc;
  return launch_gauss_pair_transitions(a, tc, 1, keep ? a.t_full : a.t_full + 1, a.sample_out,
                                       a.trace_eps, a.trace_acc, s, timer);
}

}  // namespace hmc
