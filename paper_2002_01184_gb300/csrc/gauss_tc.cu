// Dense Gaussian target on the tcgen05 tensor cores: each leapfrog step is
// one launch that computes a 128-chain x 64-column tile of the gradient
// G = -X P (a C x D x D product, Section 2.1's batched "list of vectors"
// evaluation) in 3xTF32 -- A_lo B_hi + A_hi B_lo + A_hi B_hi, float32
// accumulation in tensor memory -- and applies the leapfrog update to the
// same tile in its epilogue, so the gradient never goes to HBM.
//
// A transition (identity mass, step eps, L steps) is L + 2 launches:
//   begin:  p0 ~ N(0, I); H0 = -lp(x0) + |p0|^2/2; p = p0 + eps/2 g(x0);
//           x1 = x0 + eps p                          (cached g(x0) reused)
//   step l = 1 .. L-1:  g = -x_l P;  p += eps g;  x_{l+1} = x_l + eps p
//           (the half kicks of consecutive steps merged)
//   step L: g = -x_L P;  p += eps/2 g;  lp partials <x_L, g>/2 per tile
//   accept: H_L, Metropolis-Hastings select, traces, dual averaging
// Positions inside the trajectory are kept as their tf32 head and float32
// remainder (x = hi + lo exactly): the A operands the next product loads by
// TMA.  Both buffers are ping-ponged between steps.
//
// Tile pipeline (576 threads): warp 0 allocates tensor memory and one lane
// issues the TMA loads of the A (x hi/lo: 128 x 32) and B (P hi/lo: 64 x 32)
// K-chunks into a ring of stages; one lane of warp 1 issues the MMAs; warps
// 2-17 read the accumulator (four warps per TMEM lane quarter) and run the
// epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

constexpr int kBM = 128;          // chains per tile (MMA M)
constexpr int kBN = 64;           // output columns per tile (MMA N) of the Gaussian's products
constexpr int kBK = 32;           // K chunk: 32 floats = one 128-B swizzle row
// warp 0 TMA, warp 1 MMA, 16 epilogue warps: four per tensor-memory lane
// quarter, each moving a quarter of the tile's columns; then all sixteen walk
// the tile's rows (with four, a tile's epilogue ran one warp per SM
// sub-partition and, bound by latency, took longer than its MMAs)
constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kABytes = kBM * kBK * 4;                  // 16 KB

// A tile of BN output columns (MMA N = 64, 128 or 256): the stage ring fills
// the same 192 KB of shared memory with 4, 3 or 2 stages; the accumulator
// takes BN tensor-memory columns.  Wider tiles re-read their A operand (the
// chains' rows) fewer times: the logistic regression's products use them.
template <int BN, int ST = (BN == 64 ? 4 : BN == 128 ? 3 : 2)>
struct Tile {
  static constexpr int kStages = ST;
  // two CTAs per SM when the ring is small enough (so that one's epilogue
  // overlaps the other's products)
  static constexpr int kCtasPerSm = (BN == 64 && ST == 2) ? 2 : 1;
  static constexpr uint32_t kBBytes = BN * kBK * 4;
  static constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;
  static constexpr size_t kSmem = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kTmemCols = BN;
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  static_assert(kBM * (BN + 1) * 4 <= kStages * kStageBytes, "epilogue staging must fit the ring");
  static_assert(kSmem <= 227 * 1024, "shared memory");
};
constexpr size_t kSmemBytes = Tile<kBN>::kSmem;

// Epilogues of the tile product (the pipeline is the same for all three):
//   kEpiGauss   G = -X P: the dense Gaussian's leapfrog update
//   kEpiLrResid Z = Theta X^T (columns are data rows): R = y - sigmoid(Z)
//               to HBM as tf32 head / remainder, 0 past the last row; on
//               the last step the rows' log-likelihood terms per tile
//   kEpiStore   the raw product of K-split blockIdx.z, for a separate sum
//               (G = R X, summed with the prior and the leapfrog update by
//               k_lr_gemm_update; the dense Gaussian's X P under NUTS)
constexpr int kEpiGauss = 0, kEpiLrResid = 1, kEpiStore = 3;

struct TcStepArgs {
  int C, D;
  int ld;                   // row length of the trajectory buffers (>= D)
  int K;                    // contraction length (the Gaussian and Z: D; G: Npad)
  int ncols;                // output columns (D, or Npad for Z)
  int nvalid;               // Z: data rows N (R = 0 for columns >= N)
  const float* y;           // Z: labels [Npad]
  float* rhi;               // Z: R head / remainder [C x ldr]
  float* rlo;
  int ldr;
  int lp_col0;              // lp_part column of this product's first tile
  int kc_split;             // kEpiStore: K-chunks per split (split = blockIdx.z)
  float* part;              // kEpiStore: [splits x C x ld] products
  int last;                 // 0: middle step, 1: final step of the trajectory
  const float* xhi_in;      // x_l split (this tile's elements are re-read here)
  const float* xlo_in;
  float* xhi_out;           // x_{l+1} split (middle steps)
  float* xlo_out;
  float* p;                 // momentum, updated in place
  float* g_out;             // final step: gradient at x_L
  float* lp_part;           // final step: [C x ntn] tile partials of log p
  int ntn;                  // lp_part row stride
  const DAState* da;
  int* err;                 // set to 1 if a bounded wait gave up
  const uint8_t* active;    // null, or per-chain flags: a tile with none set is skipped
};

template <int EPI, int BN = kBN, int ST = Tile<BN>::kStages>
__global__ void __launch_bounds__(kThreads, Tile<BN, ST>::kCtasPerSm)
k_gauss_tc_step(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                TcStepArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  using T = Tile<BN, ST>;
  constexpr int kStages = T::kStages;
  constexpr uint32_t kBBytes = T::kBBytes;
  constexpr uint32_t kStageBytes = T::kStageBytes;
  constexpr uint32_t kTmemCols = T::kTmemCols;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  if (a.active) {
    // NUTS: a tile whose chains have all finished their trees has no work
    const int r = threadIdx.x;
    const bool mine = r < kBM && m0 + r < a.C && a.active[m0 + r] != 0;
    if (!__syncthreads_or(mine)) return;
  }
  const int nk_all = (a.K + kBK - 1) / kBK;
  const int kc0 = EPI == kEpiStore ? static_cast<int>(blockIdx.z) * a.kc_split : 0;
  const int nk = EPI == kEpiStore ? min(a.kc_split, nk_all - kc0) : nk_all;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(acc_full, 1);
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mAhi);
    ptx::prefetch_tensormap(&mAlo);
    ptx::prefetch_tensormap(&mBhi);
    ptx::prefetch_tensormap(&mBlo);
  }
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kStages, round = kc / kStages;
      if (kc >= kStages && !ptx::mbar_wait(&empty[s], (round - 1) & 1)) {
        atomicExch(a.err, 1);
        break;
      }
      uint8_t* st = smem + s * kStageBytes;
      ptx::mbar_arrive_expect_tx(&full[s], kStageBytes);
      const int kx = (kc0 + kc) * kBK;
      ptx::tma_load_2d(st, &mAhi, &full[s], kx, m0);
      ptx::tma_load_2d(st + kABytes, &mAlo, &full[s], kx, m0);
      ptx::tma_load_2d(st + 2 * kABytes, &mBhi, &full[s], kx, n0);
      ptx::tma_load_2d(st + 2 * kABytes + kBBytes, &mBlo, &full[s], kx, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t idesc = ptx::idesc_tf32(kBM, BN);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kStages, round = kc / kStages;
      if (!ptx::mbar_wait(&full[s], round & 1)) {
        atomicExch(a.err, 1);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t st = ptx::smem_u32(smem + s * kStageBytes);
#pragma unroll
      for (int j = 0; j < kBK / 8; ++j) {           // K = 8 tf32 per MMA (32 B)
        const uint64_t a_hi = ptx::sw128_kmajor_desc(st + 32 * j);
        const uint64_t a_lo = ptx::sw128_kmajor_desc(st + kABytes + 32 * j);
        const uint64_t b_hi = ptx::sw128_kmajor_desc(st + 2 * kABytes + 32 * j);
        const uint64_t b_lo = ptx::sw128_kmajor_desc(st + 2 * kABytes + kBBytes + 32 * j);
        ptx::mma_tf32(tmem, a_lo, b_hi, idesc, (kc | j) != 0 ? 1u : 0u);
        ptx::mma_tf32(tmem, a_hi, b_lo, idesc, 1u);
        ptx::mma_tf32(tmem, a_hi, b_hi, idesc, 1u);
      }
      ptx::mma_commit(&empty[s]);
    }
    ptx::mma_commit(acc_full);
  } else if (warp >= 2) {
    // ---- epilogue.  (1) each warp moves its 32 TMEM lanes (tile rows) into a
    // padded shared-memory tile -- the pipeline's stage buffers are free once
    // the last MMA has completed; (2) the four warps walk the tile row by row
    // with lanes along the columns, so every global access is a coalesced
    // 128-byte row segment.
    const bool ok = ptx::mbar_wait(acc_full, 0);
    if (!ok) atomicExch(a.err, 1);
    ptx::tc_fence_after();
    const int quarter = warp & 3;
    const int cgroup = (warp - 2) >> 2;               // which quarter of the columns
    float* stg = reinterpret_cast<float*>(smem);
    constexpr int kLd = BN + 1;
    constexpr int kCols = BN / 4;                     // 16, 32 or 64 per warp
#pragma unroll
    for (int c0 = cgroup * kCols; c0 < (cgroup + 1) * kCols; c0 += 16) {
      float acc[16];
      ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c0, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) stg[(quarter * 32 + lane) * kLd + c0 + j] = acc[j];
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
    const float eps = a.da->eps;
    const float* __restrict__ xhi_in = a.xhi_in;
    const float* __restrict__ xlo_in = a.xlo_in;
    float* __restrict__ xhi_out = a.xhi_out;
    float* __restrict__ xlo_out = a.xlo_out;
    float* __restrict__ pm = a.p;
    float* __restrict__ g_out = a.g_out;
    const int ew = warp - 2;
#pragma unroll 2
    for (int rr = 0; rr < kBM / kEpiWarps; ++rr) {
      const int r = ew + kEpiWarps * rr;
      const int m = m0 + r;
      if (!ok || m >= a.C) continue;                  // warp-uniform
      float part = 0.f;
      if (EPI == kEpiStore) {
        float* out = a.part + (static_cast<int64_t>(blockIdx.z) * a.C + m) * a.ld;
#pragma unroll
        for (int h = 0; h < BN / 32; ++h) {
          const int n = n0 + lane + 32 * h;
          if (n < a.D) out[n] = stg[r * kLd + lane + 32 * h];
        }
        continue;
      }
      if (EPI == kEpiLrResid) {
        const int64_t rowoff = static_cast<int64_t>(m) * a.ldr;
#pragma unroll
        for (int h = 0; h < BN / 32; ++h) {
          const int cl = lane + 32 * h;
          const int n = n0 + cl;
          if (n < a.ncols) {
            float res = 0.f;
            if (n < a.nvalid) {
              const float z = stg[r * kLd + cl];
              const float yv = a.y[n];
              res = residual_f(yv, z);
              if (a.last) part += loglik_f(yv, z);
            }
            float hi, lo;
            split_tf32(res, hi, lo);
            a.rhi[rowoff + n] = hi;
            a.rlo[rowoff + n] = lo;
          }
        }
      } else {
        const int64_t rowoff = static_cast<int64_t>(m) * a.ld;
#pragma unroll
        for (int h = 0; h < BN / 32; ++h) {
          const int cl = lane + 32 * h;
          const int n = n0 + cl;
          if (n < a.D) {
            const int64_t e = rowoff + n;
            const float x = xhi_in[e] + xlo_in[e];
            const float g = -stg[r * kLd + cl];
            if (!a.last) {
              const float p = fmaf(eps, g, pm[e]);
              pm[e] = p;
              float hi, lo;
              split_tf32(fmaf(eps, p, x), hi, lo);
              xhi_out[e] = hi;
              xlo_out[e] = lo;
            } else {
              pm[e] = fmaf(0.5f * eps, g, pm[e]);
              g_out[e] = g;
              part = fmaf(x, g, part);
            }
          }
        }
      }
      if (a.last) {
        part = warp_sum(part);
        // Gaussian: log p = <x, g> / 2; logistic regression: the rows'
        // log-likelihood terms, or the prior's -|theta|^2 / 2
        const float v = EPI == kEpiLrResid ? part : 0.5f * part;
        if (lane == 0) a.lp_part[static_cast<int64_t>(m) * a.ntn + a.lp_col0 + blockIdx.y] = v;
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
}

// Z = Theta X^T with the residual epilogue as one persistent launch (the
// leapfrog steps of HMC; NUTS, which skips tiles whose chains have finished,
// keeps k_gauss_tc_step).  One CTA per SM takes tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... of 128 chains x 64 data rows; the TMA ring runs
// on across its tiles and the accumulator is double-buffered in tensor
// memory, so the MMAs of one tile run while the epilogue turns the previous
// tile's Z into R.  The four warps of a tensor-memory lane quarter each
// compute 16 columns of its 32 rows, stage them in the quarter's shared
// rows, meet, and store 8 whole rows each (128-byte stores).  (One tile per
// CTA left each CTA's ring fill, MMAs and epilogue in sequence; a persistent
// form whose threads stored their own row's columns was bound by those
// scattered stores.)
constexpr int kZpStages = 3;
constexpr int kZpBN = 64;                               // data rows per tile
constexpr uint32_t kZpABytes = kBM * kBK * 4;          // 16 KB: 128 chains x 32 dims
constexpr uint32_t kZpBBytes = kZpBN * kBK * 4;        // 8 KB: 64 data rows x 32 dims
constexpr uint32_t kZpStage = 2 * kZpABytes + 2 * kZpBBytes;
constexpr int kZpLd = kZpBN + 1;                       // staged row stride (floats)
constexpr uint32_t kZpStgBytes = 4 * 2 * 32 * kZpLd * 4;   // [quarter][hi, lo][32 rows][kZpLd]
// ring, staging, log-likelihood partials [4 column groups][128 rows],
// barriers and tensor-memory slot, alignment slack
constexpr size_t kZpSmem = kZpStages * kZpStage + kZpStgBytes + 4 * kBM * 4 + 256 + 1024;
static_assert(kZpSmem <= 227 * 1024, "shared memory");
static_assert(8 * (2 * kZpStages + 4) + 16 <= 256, "barriers");
static_assert(kEpiWarps == 16 && kZpBN == 4 * 16, "four column groups of 16 per lane quarter");

__global__ void __launch_bounds__(kThreads, 1)
k_lr_z_persist(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
               const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
               TcStepArgs a, int mt, int ntiles) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float* stg = reinterpret_cast<float*>(smem + kZpStages * kZpStage);           // staging
  float* lps = stg + kZpStgBytes / 4;                                          // [4][kBM]
  uint64_t* full = reinterpret_cast<uint64_t*>(lps + 4 * kBM);
  uint64_t* empty = full + kZpStages;
  uint64_t* acc_full = empty + kZpStages;      // [2]
  uint64_t* acc_empty = acc_full + 2;          // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (a.K + kBK - 1) / kBK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kZpStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], 32 * kEpiWarps);
    }
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mAhi);
    ptx::prefetch_tensormap(&mAlo);
    ptx::prefetch_tensormap(&mBhi);
    ptx::prefetch_tensormap(&mBlo);
  }
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, 2 * kZpBN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // tile t: chains (t % mt) 128, data rows (t / mt) 64
  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one ring across all of this CTA's tiles
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int m0 = (t % mt) * kBM, n0 = (t / mt) * kZpBN;
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int s = it % kZpStages, round = it / kZpStages;
        if (it >= kZpStages && !ptx::mbar_wait(&empty[s], (round - 1) & 1)) {
          atomicExch(a.err, 1);
          ok = false;
          break;
        }
        uint8_t* st = smem + s * kZpStage;
        ptx::mbar_arrive_expect_tx(&full[s], kZpStage);
        const int kx = kc * kBK;
        ptx::tma_load_2d(st, &mAhi, &full[s], kx, m0);
        ptx::tma_load_2d(st + kZpABytes, &mAlo, &full[s], kx, m0);
        ptx::tma_load_2d(st + 2 * kZpABytes, &mBhi, &full[s], kx, n0);
        ptx::tma_load_2d(st + 2 * kZpABytes + kZpBBytes, &mBlo, &full[s], kx, n0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: tile k into accumulator buffer k % 2, once the
    // epilogue has read that buffer's previous tile
    constexpr uint32_t idesc = ptx::idesc_tf32(kBM, kZpBN);
    int it = 0, k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++k) {
      const int b = k & 1;
      if (k >= 2 && !ptx::mbar_wait(&acc_empty[b], ((k >> 1) - 1) & 1)) {
        atomicExch(a.err, 1);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t acc = tmem + static_cast<uint32_t>(kZpBN * b);
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int s = it % kZpStages, round = it / kZpStages;
        if (!ptx::mbar_wait(&full[s], round & 1)) {
          atomicExch(a.err, 1);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t st = ptx::smem_u32(smem + s * kZpStage);
#pragma unroll
        for (int j = 0; j < kBK / 8; ++j) {
          const uint64_t a_hi = ptx::sw128_kmajor_desc(st + 32 * j);
          const uint64_t a_lo = ptx::sw128_kmajor_desc(st + kZpABytes + 32 * j);
          const uint64_t b_hi = ptx::sw128_kmajor_desc(st + 2 * kZpABytes + 32 * j);
          const uint64_t b_lo = ptx::sw128_kmajor_desc(st + 2 * kZpABytes + kZpBBytes + 32 * j);
          ptx::mma_tf32(acc, a_lo, b_hi, idesc, (kc | j) != 0 ? 1u : 0u);
          ptx::mma_tf32(acc, a_hi, b_lo, idesc, 1u);
          ptx::mma_tf32(acc, a_hi, b_hi, idesc, 1u);
        }
        ptx::mma_commit(&empty[s]);
      }
      if (ok) ptx::mma_commit(&acc_full[b]);
    }
  } else if (warp >= 2) {
    // ---- epilogue: warp (quarter q, column group cg) computes columns
    // 16 cg .. 16 cg + 15 of rows 32 q .. 32 q + 31 (thread = row), stages
    // them, and after the quarter's barrier stores rows 8 cg .. 8 cg + 7
    // whole (two 128-byte stores per row and array)
    const int quarter = warp & 3, cg = (warp - 2) >> 2;
    float* qh = stg + quarter * 2 * 32 * kZpLd;      // the quarter's staged R head
    float* ql = qh + 32 * kZpLd;                      // and remainder
    const uint32_t qbar = 2u + static_cast<uint32_t>(quarter);   // named barrier of the quarter's 4 warps
    bool bad = false;              // a wait gave up: later tiles skip their waits and stores
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int b = k & 1;
      const int m0 = (t % mt) * kBM, n0 = (t / mt) * kZpBN, n = n0 + 16 * cg;
      const int m = m0 + quarter * 32 + lane;
      if (!bad && !ptx::mbar_wait(&acc_full[b], (k >> 1) & 1)) {
        atomicExch(a.err, 1);
        bad = true;
      }
      ptx::tc_fence_after();
      float v[16];
      ptx::tmem_ld16(tmem + static_cast<uint32_t>(kZpBN * b + 16 * cg) + (static_cast<uint32_t>(quarter * 32) << 16),
                     v);
      ptx::tc_fence_before();
      ptx::mbar_arrive_local(&acc_empty[b]);
      // R = y - sigmoid(Z) for the 16 columns (labels the same for every lane)
      float yv[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 u = reinterpret_cast<const float4*>(a.y + n)[q];
        yv[4 * q] = u.x; yv[4 * q + 1] = u.y; yv[4 * q + 2] = u.z; yv[4 * q + 3] = u.w;
      }
      float part = 0.f;
      // the quarter's staged rows of the previous tile are stored: restage
      if (k > 0) asm volatile("bar.sync %0, 128;" ::"r"(qbar) : "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float res = 0.f;
        if (n + j < a.nvalid) {
          res = residual_f(yv[j], v[j]);
          if (a.last) part += loglik_f(yv[j], v[j]);
        }
        float hi, lo;
        split_tf32(res, hi, lo);
        qh[lane * kZpLd + 16 * cg + j] = hi;
        ql[lane * kZpLd + 16 * cg + j] = lo;
      }
      if (a.last) lps[cg * kBM + quarter * 32 + lane] = part;
      asm volatile("bar.sync %0, 128;" ::"r"(qbar) : "memory");
      if (!bad) {
        // rows 8 cg .. 8 cg + 7 of the quarter, lanes along the columns
#pragma unroll 2
        for (int rr = 8 * cg; rr < 8 * cg + 8; ++rr) {
          const int mr = m0 + quarter * 32 + rr;
          if (mr >= a.C) continue;                    // warp-uniform
          float* oh = a.rhi + static_cast<int64_t>(mr) * a.ldr + n0;
          float* ol = a.rlo + static_cast<int64_t>(mr) * a.ldr + n0;
          oh[lane] = qh[rr * kZpLd + lane];
          oh[lane + 32] = qh[rr * kZpLd + lane + 32];
          ol[lane] = ql[rr * kZpLd + lane];
          ol[lane + 32] = ql[rr * kZpLd + lane + 32];
        }
        // the rows' log-likelihood terms: the four column groups in order
        if (a.last && cg == 0 && m < a.C) {
          const float* l = lps + quarter * 32 + lane;
          a.lp_part[static_cast<int64_t>(m) * a.ntn + a.lp_col0 + t / mt] =
              ((l[0] + l[kBM]) + l[2 * kBM]) + l[3 * kBM];
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 2 * kZpBN);
  }
}

constexpr int kWarpsPerBlock = 8;

struct TcBeginAccept {
  StepArgs s;
  int ld;            // row length of p, xhi, xlo, gL (>= D; the state x, g has rows of D)
  float* p;
  float* xhi;        // begin: x1 split out; accept: x_L split in
  float* xlo;
  float* gL;
  float* lp_part;
  float* h0;
  int ntn;
};

// p0 ~ N(0, I); H0; half kick with the cached gradient; first drift (warp per chain)
__global__ void k_gauss_tc_begin(TcBeginAccept b) {
  const StepArgs& a = b.s;
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.C) return;
  const int D = a.D;
  const int64_t row = static_cast<int64_t>(c) * D, rowi = static_cast<int64_t>(c) * b.ld;
  const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
  const float eps = a.da->eps;
  float kin = 0.f;
  for (int j = lane; 4 * j < D; j += 32) {
    const float4 z = momentum4(a.seed, static_cast<uint32_t>(j), chain, a.t);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int i = 0; i < 4 && 4 * j + i < D; ++i) {
      const int64_t e = row + 4 * j + i, ei = rowi + 4 * j + i;
      kin = fmaf(zz[i], zz[i], kin);
      const float p = fmaf(0.5f * eps, a.g[e], zz[i]);
      b.p[ei] = p;
      float hi, lo;
      split_tf32(fmaf(eps, p, a.x[e]), hi, lo);
      b.xhi[ei] = hi;
      b.xlo[ei] = lo;
    }
  }
  kin = warp_sum(kin);
  if (lane == 0) b.h0[c] = -a.lp[c] + 0.5f * kin;
}

// H_L from the tile partials and |p|^2; Metropolis-Hastings select; traces;
// dual averaging (warp per chain)
__global__ void k_gauss_tc_accept(TcBeginAccept b) {
  const StepArgs& a = b.s;
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) {
    const int D = a.D;
    const int64_t row = static_cast<int64_t>(c) * D, rowi = static_cast<int64_t>(c) * b.ld;
    const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
    float kin = 0.f;
    for (int d = lane; d < D; d += 32) kin = fmaf(b.p[rowi + d], b.p[rowi + d], kin);
    kin = 0.5f * warp_sum(kin);
    float lp1 = 0.f;
    if (lane == 0)
      for (int k = 0; k < b.ntn; ++k) lp1 += b.lp_part[static_cast<int64_t>(c) * b.ntn + k];
    lp1 = __shfl_sync(0xffffffffu, lp1, 0);
    float la = b.h0[c] - (-lp1 + kin);
    if (!isfinite(la)) la = -INFINITY;
    int acc = 0;
    if (lane == 0) acc = accept_log_uniform(a.seed, chain, a.t) < la;
    acc = __shfl_sync(0xffffffffu, acc, 0);
    for (int d = lane; d < D; d += 32) {
      const int64_t e = row + d, ei = rowi + d;
      if (acc) {
        a.x[e] = b.xhi[ei] + b.xlo[ei];
        a.g[e] = b.gL[ei];
      }
      if (a.sample_out) a.sample_out[e] = a.x[e];
    }
    if (lane == 0) {
      if (acc) a.lp[c] = lp1;
      a.is_accepted[c] = static_cast<uint8_t>(acc);
      a.log_accept[c] = la;
      if (a.trace_acc) a.trace_acc[c] = static_cast<uint8_t>(acc);
      if (c == 0 && a.trace_eps) a.trace_eps[0] = a.da->eps;
    }
    prob = accept_prob(la);
  }
  accept_block_finish<kWarpsPerBlock>(a.da, a.partials, prob, has_chain, a.C, a.t_full);
}

// The logistic regression's split-K gradient: the splits' products summed in
// split order, minus theta (the prior), and the leapfrog update.  Warp per
// chain, four dims per lane (ld % 4 == 0; the library's own buffers).
struct LrSumArgs {
  int C, D, ld, S, last, nrt, ntot;
  const float* part;        // [S x C x ld]
  const float* xhi_in;
  const float* xlo_in;
  float* xhi_out;
  float* xlo_out;
  float* p;
  float* g_out;
  float* lp_part;
  const DAState* da;
};

__global__ void k_lr_gemm_update(LrSumArgs b) {
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= b.C) return;
  const int ld4 = b.ld >> 2;
  const int64_t row4 = static_cast<int64_t>(c) * ld4, split4 = static_cast<int64_t>(b.C) * ld4;
  const float eps = b.da->eps;
  const float4* part = reinterpret_cast<const float4*>(b.part);
  float sq = 0.f;
  for (int j = lane; j < ld4; j += 32) {
    const int64_t e = row4 + j;
    const float4 h = reinterpret_cast<const float4*>(b.xhi_in)[e];
    const float4 l = reinterpret_cast<const float4*>(b.xlo_in)[e];
    const float th[4] = {h.x + l.x, h.y + l.y, h.z + l.z, h.w + l.w};
    float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int sp = 0; sp < b.S; ++sp) {
      const float4 v = part[sp * split4 + e];
      g[0] += v.x; g[1] += v.y; g[2] += v.z; g[3] += v.w;
    }
    const float4 pv = reinterpret_cast<float4*>(b.p)[e];
    const float pin[4] = {pv.x, pv.y, pv.z, pv.w};
    float pout[4], hi[4], lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // padding dims (>= D) hold zeros everywhere and stay zero
      g[k] = 4 * j + k < b.D ? g[k] - th[k] : 0.f;
      if (!b.last) {
        pout[k] = fmaf(eps, g[k], pin[k]);
        split_tf32(fmaf(eps, pout[k], th[k]), hi[k], lo[k]);
      } else {
        pout[k] = fmaf(0.5f * eps, g[k], pin[k]);
        sq = fmaf(th[k], th[k], sq);
      }
    }
    reinterpret_cast<float4*>(b.p)[e] = make_float4(pout[0], pout[1], pout[2], pout[3]);
    if (!b.last) {
      reinterpret_cast<float4*>(b.xhi_out)[e] = make_float4(hi[0], hi[1], hi[2], hi[3]);
      reinterpret_cast<float4*>(b.xlo_out)[e] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    } else {
      reinterpret_cast<float4*>(b.g_out)[e] = make_float4(g[0], g[1], g[2], g[3]);
    }
  }
  if (b.last) {
    sq = warp_sum(sq);
    // the prior's -|theta|^2 / 2 in the first prior column, the others zero
    for (int k = lane; k < b.ntot - b.nrt; k += 32)
      b.lp_part[static_cast<int64_t>(c) * b.ntot + b.nrt + k] = k == 0 ? -0.5f * sq : 0.f;
  }
}

// P -> (tf32 head, float32 remainder)
__global__ void k_split(int64_t n, const float* __restrict__ src, float* __restrict__ hi,
                        float* __restrict__ lo) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float h, l;
    split_tf32(src[i], h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Row-major [rows x cols] float32 matrix, box of 32 columns x box_rows rows,
// 128-byte swizzle (matches sw128_kmajor_desc).
bool make_map(CUtensorMap* map, const float* base, int64_t rows, int cols, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * sizeof(float)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

// [K x C x D] float32 samples as a 3-D tensor (D innermost), box of 128 dims x
// 64 chains x 1 sample, no swizzle: the layout of a [64][128] row-major tile.
bool make_sample_map(CUtensorMap* map, const float* base, int D, int64_t C, int64_t K) {
  auto fn = encode_fn();
  if (!fn || D % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0 || C < 1 || K < 1) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(D), static_cast<cuuint64_t>(C), static_cast<cuuint64_t>(K)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(D) * sizeof(float),
                           static_cast<cuuint64_t>(C) * static_cast<cuuint64_t>(D) * sizeof(float)};
  cuuint32_t box[3] = {128, 64, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

inline unsigned blocks_for(int64_t n) {
  return static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 152 * 16));
}

}  // namespace

bool gauss_tc_supported(const hmc_target& t) {
  return t.id == HMC_T_CORR_GAUSS && t.dim % 4 == 0 && encode_fn() != nullptr;
}

size_t gauss_tc_workspace_bytes(const hmc_target& t, int64_t C) {
  const size_t CD = static_cast<size_t>(C) * t.dim, DD = static_cast<size_t>(t.dim) * t.dim;
  const size_t ntn = (t.dim + kBN - 1) / kBN;
  auto a = [](size_t b) { return (b + 1023) & ~static_cast<size_t>(1023); };
  const size_t image = t.dim <= 256 ? a(kGaussPairImageFloats * 4) : 0;
  const size_t blocks = t.dim <= 256 ? 6 * a(static_cast<size_t>(gauss_pair_padded_chains(C)) * t.dim * 4) + a(24) : 0;
  return 2 * a(DD * 4) + 6 * a(CD * 4) + a(C * ntn * 4) + a(C * 4) + a(sizeof(int)) + image + blocks;
}

cudaError_t gauss_tc_setup(GaussTc* tc, const hmc_target& t, int64_t C, void* ws, cudaStream_t s) {
  const size_t CD = static_cast<size_t>(C) * t.dim, DD = static_cast<size_t>(t.dim) * t.dim;
  auto a = [](size_t b) { return (b + 1023) & ~static_cast<size_t>(1023); };
  char* w = static_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* p = w; w += a(bytes); return reinterpret_cast<float*>(p); };
  tc->ntn = (t.dim + kBN - 1) / kBN;
  tc->Phi = take(DD * 4);
  tc->Plo = take(DD * 4);
  for (int i = 0; i < 2; ++i) {
    tc->xhi[i] = take(CD * 4);
    tc->xlo[i] = take(CD * 4);
  }
  tc->p = take(CD * 4);
  tc->gL = take(CD * 4);
  tc->lp_part = take(C * tc->ntn * 4);
  tc->h0 = take(C * 4);
  tc->err = reinterpret_cast<int*>(take(sizeof(int)));
  tc->Ptm = t.dim <= 256 ? take(kGaussPairImageFloats * 4) : nullptr;
  if (t.dim <= 256) {
    const size_t blk = static_cast<size_t>(gauss_pair_padded_chains(C)) * t.dim * 4;
    tc->pair_g = take(blk);
    tc->pair_p = take(2 * blk);
    tc->pair_w = take(3 * blk);
    tc->pair_stat = reinterpret_cast<unsigned long long*>(take(3 * sizeof(unsigned long long)));
  }
  bool ok = make_map(&tc->mBhi, tc->Phi, t.dim, t.dim, kBN) &&
            make_map(&tc->mBlo, tc->Plo, t.dim, t.dim, kBN) &&
            make_map(&tc->mPhi128, tc->Phi, t.dim, t.dim, 128) &&
            make_map(&tc->mPlo128, tc->Plo, t.dim, t.dim, 128);
  for (int i = 0; i < 2 && ok; ++i)
    ok = make_map(&tc->mAhi[i], tc->xhi[i], C, t.dim, kBM) &&
         make_map(&tc->mAlo[i], tc->xlo[i], C, t.dim, kBM);
  if (!ok) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_gauss_tc_step<kEpiGauss>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmemBytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gauss_tc_step<kEpiStore>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmemBytes));
  if (e != cudaSuccess) return e;
  if (gauss_fused_supported(t)) {
    e = gauss_fused_setup();
    if (e == cudaSuccess) e = gauss_pair_setup();
    if (e != cudaSuccess) return e;
  }
  k_split<<<blocks_for(DD), 256, 0, s>>>(static_cast<int64_t>(DD), t.P, tc->Phi, tc->Plo);
  count_launch();
  if (tc->Ptm) {
    e = launch_gauss_pair_image(tc->Phi, tc->Plo, t.dim, tc->Ptm, s);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(tc->err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_gauss_tc_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                       KernelTimer* timer) {
  if (tc.fused && tc.pair) return launch_gauss_pair_transition(a, tc, s, timer);
  if (tc.fused) return launch_gauss_fused_transition(a, tc, s, timer);
  TcBeginAccept b{};
  b.s = a;
  b.p = tc.p;
  b.gL = tc.gL;
  b.lp_part = tc.lp_part;
  b.h0 = tc.h0;
  b.ntn = tc.ntn;
  b.ld = a.D;
  b.xhi = tc.xhi[0];
  b.xlo = tc.xlo[0];
  const unsigned nb = static_cast<unsigned>((a.C + kWarpsPerBlock - 1) / kWarpsPerBlock);
  k_gauss_tc_begin<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
  count_launch();
  const dim3 grid((a.C + kBM - 1) / kBM, tc.ntn);
  for (int l = 1; l <= a.L; ++l) {
    TcStepArgs st{};
    st.C = a.C;
    st.D = a.D;
    st.ld = a.D;
    st.K = a.D;
    st.ncols = a.D;
    st.lp_col0 = 0;
    st.last = l == a.L;
    const int in = (l - 1) & 1, out = l & 1;
    st.xhi_in = tc.xhi[in];
    st.xlo_in = tc.xlo[in];
    st.xhi_out = tc.xhi[out];
    st.xlo_out = tc.xlo[out];
    st.p = tc.p;
    st.g_out = tc.gL;
    st.lp_part = tc.lp_part;
    st.ntn = tc.ntn;
    st.da = a.da;
    st.err = tc.err;
    if (timer) timer->begin(s);
    k_gauss_tc_step<kEpiGauss><<<grid, kThreads, kSmemBytes, s>>>(tc.mAhi[in], tc.mAlo[in], tc.mBhi, tc.mBlo,
                                                                   st);
    if (timer) timer->end(s);
    count_launch();
  }
  b.xhi = tc.xhi[(a.L - 1) & 1];
  b.xlo = tc.xlo[(a.L - 1) & 1];
  k_gauss_tc_accept<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
  count_launch();
  return cudaGetLastError();
}


cudaError_t launch_gauss_tc_product(GaussTc& tc, int C, int D, const DAState* da, const uint8_t* active,
                                    cudaStream_t s) {
  TcStepArgs st{};
  st.C = C;
  st.D = D;
  st.ld = D;
  st.K = D;
  st.ncols = D;
  st.kc_split = (D + kBK - 1) / kBK;
  st.part = tc.gL;
  st.da = da;
  st.err = tc.err;
  st.active = active;
  const dim3 grid((C + kBM - 1) / kBM, tc.ntn, 1);
  k_gauss_tc_step<kEpiStore><<<grid, kThreads, kSmemBytes, s>>>(tc.mAhi[0], tc.mAlo[0], tc.mBhi, tc.mBlo, st);
  count_launch();
  return cudaGetLastError();
}


bool logreg_gemm_supported(const hmc_target& t) {
  return t.id == HMC_T_LOGREG && t.n_data >= 1 && encode_fn() != nullptr;
}

namespace {
// data rows padded to whole 64-row tiles (the residual product's columns,
// the gradient product's K)
int64_t lr_npad(int64_t n) { return (n + kBN - 1) / kBN * kBN; }
// the most K-splits of the gradient product G = R X
constexpr int kMaxSplit = 16;
size_t a1k(size_t b) { return (b + 1023) & ~static_cast<size_t>(1023); }

// Tile widths: Z = Theta X^T in 64-row tiles of the data with a 2-stage ring
// (96 KB), so that two CTAs share an SM and one's epilogue (the residual,
// R to HBM) overlaps the other's products -- 128-row tiles at one CTA per SM
// measured 5 % slower on a dim-254, 19102-row, 1204-chain gradient; G = R X
// in one tile over the dims up to 256 wide (each re-reads R, C x Npad, from
// HBM: four times at 64 columns for a dim of 256)
struct LrTiles {
  int bnz, bng, nrt, ndt;
};
template <int EPI>
void launch_tile(int bn, dim3 grid, const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc,
                 const CUtensorMap& md, const TcStepArgs& st, cudaStream_t s) {
  if (bn == 64)
    k_gauss_tc_step<EPI, 64><<<grid, kThreads, Tile<64>::kSmem, s>>>(ma, mb, mc, md, st);
  else if (bn == 128)
    k_gauss_tc_step<EPI, 128><<<grid, kThreads, Tile<128>::kSmem, s>>>(ma, mb, mc, md, st);
  else
    k_gauss_tc_step<EPI, 256><<<grid, kThreads, Tile<256>::kSmem, s>>>(ma, mb, mc, md, st);
}

LrTiles lr_tiles(int64_t npad, int ld) {
  LrTiles q{};
  q.bnz = 64;
  q.bng = ld <= 64 ? 64 : ld <= 128 ? 128 : 256;
  q.nrt = static_cast<int>((npad + q.bnz - 1) / q.bnz);
  q.ndt = (ld + q.bng - 1) / q.bng;
  return q;
}

// G = R X has K = Npad but only (C / 128) x ndt tiles: split K when the tiles
// would not fill two waves of the SMs, and sum the splits afterwards
void lr_splits(const LogregGemm& g, int C, int* S_out, int* kc_out) {
  const int64_t mt = (C + kBM - 1) / kBM;
  const int nk_all = g.npad / kBK;
  const int64_t tiles = mt * g.ndt;
  int S = 1, kc_split = nk_all;
  const int64_t sms = g.sms;
  if (tiles < 2 * sms && nk_all >= 2) {
    S = static_cast<int>(std::min<int64_t>({kMaxSplit, (2 * sms + tiles - 1) / tiles, nk_all}));
    kc_split = (nk_all + S - 1) / S;
    S = (nk_all + kc_split - 1) / kc_split;      // every split has at least one chunk
  }
  *S_out = S;
  *kc_out = kc_split;
}
}  // namespace

size_t logreg_gemm_workspace_bytes(const hmc_target& t, int64_t C) {
  const size_t npad = static_cast<size_t>(lr_npad(t.n_data)), D = static_cast<size_t>((t.dim + 3) / 4 * 4);
  const size_t ND = npad * D, CN = static_cast<size_t>(C) * npad, CD = static_cast<size_t>(C) * D;
  const LrTiles q = lr_tiles(static_cast<int64_t>(npad), static_cast<int>(D));
  const size_t ntot = static_cast<size_t>(q.nrt + q.ndt);
  return 4 * a1k(ND * 4) + a1k(npad * 4) + 2 * a1k(CN * 4) + 6 * a1k(CD * 4) +
         a1k(static_cast<size_t>(C) * ntot * 4) + a1k(static_cast<size_t>(C) * 4) + a1k(sizeof(int)) +
         a1k(kMaxSplit * CD * 4);
}

cudaError_t logreg_gemm_setup(LogregGemm* g, const hmc_target& t, int64_t C, void* ws, cudaStream_t s) {
  const int64_t npad = lr_npad(t.n_data);
  const int ld = (t.dim + 3) / 4 * 4;      // rows padded for the 16-byte TMA strides
  const size_t D = static_cast<size_t>(ld);
  const size_t ND = static_cast<size_t>(npad) * D, CN = static_cast<size_t>(C) * npad,
               CD = static_cast<size_t>(C) * D;
  g->npad = static_cast<int>(npad);
  g->nvalid = static_cast<int>(t.n_data);
  g->ld = ld;
  int dev = 0;
  cudaError_t qe = cudaGetDevice(&dev);
  if (qe == cudaSuccess) qe = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
  if (qe != cudaSuccess) return qe;
  const LrTiles q = lr_tiles(npad, ld);
  g->bnz = q.bnz;
  g->bng = q.bng;
  g->nrt = q.nrt;
  g->ndt = q.ndt;
  g->ntot = g->nrt + g->ndt;
  char* w = static_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* q = w; w += a1k(bytes); return reinterpret_cast<float*>(q); };
  g->Xhi = take(ND * 4);
  g->Xlo = take(ND * 4);
  g->XThi = take(ND * 4);
  g->XTlo = take(ND * 4);
  g->ypad = take(static_cast<size_t>(npad) * 4);
  g->Rhi = take(CN * 4);
  g->Rlo = take(CN * 4);
  for (int i = 0; i < 2; ++i) {
    g->xhi[i] = take(CD * 4);
    g->xlo[i] = take(CD * 4);
  }
  g->p = take(CD * 4);
  g->gL = take(CD * 4);
  g->lp_part = take(static_cast<size_t>(C) * g->ntot * 4);
  g->h0 = take(static_cast<size_t>(C) * 4);
  g->err = reinterpret_cast<int*>(take(sizeof(int)));
  g->part = take(kMaxSplit * CD * 4);
  // (a box may be taller than the array: the rows past its end load as zeros)
  bool ok = make_map(&g->mXhi, g->Xhi, npad, ld, q.bnz) && make_map(&g->mXlo, g->Xlo, npad, ld, q.bnz) &&
            make_map(&g->mRhi, g->Rhi, C, static_cast<int>(npad), kBM) &&
            make_map(&g->mRlo, g->Rlo, C, static_cast<int>(npad), kBM) &&
            make_map(&g->mXThi, g->XThi, ld, static_cast<int>(npad), q.bng) &&
            make_map(&g->mXTlo, g->XTlo, ld, static_cast<int>(npad), q.bng);
  for (int i = 0; i < 2 && ok; ++i)
    ok = make_map(&g->mThi[i], g->xhi[i], C, ld, kBM) && make_map(&g->mTlo[i], g->xlo[i], C, ld, kBM);
  if (!ok) return cudaErrorInvalidValue;
  static_assert(kZpBN == 64, "the data tensor maps' box is 64 rows (lr_tiles)");
  cudaError_t e = cudaFuncSetAttribute(k_gauss_tc_step<kEpiLrResid, 64, 2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Tile<64, 2>::kSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lr_z_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kZpSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gauss_tc_step<kEpiStore, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Tile<64>::kSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gauss_tc_step<kEpiStore, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Tile<128>::kSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gauss_tc_step<kEpiStore, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Tile<256>::kSmem));
  if (e == cudaSuccess)
    e = launch_lr_prepare(static_cast<int>(t.n_data), static_cast<int>(npad), t.dim, ld, t.X, t.y, g->Xhi,
                          g->Xlo, g->XThi, g->XTlo, g->ypad, s);
  // the padding columns of the trajectory buffers are read as operands but
  // never written: zero once (the workspace is contiguous from xhi[0] to gL)
  if (e == cudaSuccess)
    e = cudaMemsetAsync(g->xhi[0], 0, reinterpret_cast<char*>(g->gL) + a1k(CD * 4) -
                                          reinterpret_cast<char*>(g->xhi[0]), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->err, 0, sizeof(int), s);
  return e;
}


// begin; L x (Z = Theta X^T with the residual epilogue, then G = R X with
// the prior and the leapfrog update); accept.  The timer brackets one
// gradient (both products).
cudaError_t launch_logreg_gemm_transition(const StepArgs& a, LogregGemm& g, cudaStream_t s,
                                          KernelTimer* timer) {
  TcBeginAccept b{};
  b.s = a;
  b.p = g.p;
  b.gL = g.gL;
  b.lp_part = g.lp_part;
  b.h0 = g.h0;
  b.ntn = g.ntot;
  b.ld = g.ld;
  b.xhi = g.xhi[0];
  b.xlo = g.xlo[0];
  const unsigned nb = static_cast<unsigned>((a.C + kWarpsPerBlock - 1) / kWarpsPerBlock);
  k_gauss_tc_begin<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
  count_launch();
  const unsigned mt = static_cast<unsigned>((a.C + kBM - 1) / kBM);
  int S = 1, kc_split = 1;
  lr_splits(g, a.C, &S, &kc_split);
  for (int l = 1; l <= a.L; ++l) {
    const int in = (l - 1) & 1, out = l & 1;
    const bool last = l == a.L;
    TcStepArgs z{};
    z.C = a.C;
    z.D = a.D;
    z.ld = g.ld;
    z.K = g.ld;
    z.ncols = g.npad;
    z.nvalid = g.nvalid;
    z.y = g.ypad;
    z.rhi = g.Rhi;
    z.rlo = g.Rlo;
    z.ldr = g.npad;
    z.lp_col0 = 0;
    z.last = last;
    z.lp_part = g.lp_part;
    z.ntn = g.ntot;
    z.da = a.da;
    z.err = g.err;
    TcStepArgs st{};
    st.C = a.C;
    st.D = a.D;
    st.ld = g.ld;
    st.K = g.npad;
    st.ncols = a.D;
    st.last = last;
    st.xhi_in = g.xhi[in];
    st.xlo_in = g.xlo[in];
    st.xhi_out = g.xhi[out];
    st.xlo_out = g.xlo[out];
    st.p = g.p;
    st.g_out = g.gL;
    st.lp_part = g.lp_part;
    st.ntn = g.ntot;
    st.lp_col0 = g.nrt;
    st.da = a.da;
    st.err = g.err;
    if (timer) timer->begin(s);
    {
      const int zt = static_cast<int>(mt) * g.nrt;      // Z tiles, one persistent CTA per SM
      k_lr_z_persist<<<static_cast<unsigned>(std::min(zt, g.sms)), kThreads, kZpSmem, s>>>(
          g.mThi[in], g.mTlo[in], g.mXhi, g.mXlo, z, static_cast<int>(mt), zt);
    }
    {
      // the split products G = R X, then their sum with the prior and the
      // leapfrog update (k_lr_gemm_update)
      st.kc_split = kc_split;
      st.part = g.part;
      launch_tile<kEpiStore>(g.bng, dim3(mt, g.ndt, S), g.mRhi, g.mRlo, g.mXThi, g.mXTlo, st, s);
      LrSumArgs u{a.C, a.D, g.ld, S, last ? 1 : 0, g.nrt, g.ntot, g.part, g.xhi[in], g.xlo[in],
                  g.xhi[out], g.xlo[out], g.p, g.gL, g.lp_part, a.da};
      k_lr_gemm_update<<<nb, 32 * kWarpsPerBlock, 0, s>>>(u);
      count_launch();
    }
    if (timer) timer->end(s);
    count_launch(2);
  }
  b.xhi = g.xhi[(a.L - 1) & 1];
  b.xlo = g.xlo[(a.L - 1) & 1];
  k_gauss_tc_accept<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_logreg_gemm_products(LogregGemm& g, int C, int D, const DAState* da,
                                        const uint8_t* active, int* splits, cudaStream_t s) {
  const unsigned mt = static_cast<unsigned>((C + kBM - 1) / kBM);
  int S = 1, kc_split = 1;
  lr_splits(g, C, &S, &kc_split);
  TcStepArgs z{};
  z.C = C;
  z.D = D;
  z.ld = g.ld;
  z.K = g.ld;
  z.ncols = g.npad;
  z.nvalid = g.nvalid;
  z.y = g.ypad;
  z.rhi = g.Rhi;
  z.rlo = g.Rlo;
  z.ldr = g.npad;
  z.lp_col0 = 0;
  z.last = 1;                  // the rows' log-likelihood partials: log p at every leaf
  z.lp_part = g.lp_part;
  z.ntn = g.ntot;
  z.da = da;
  z.err = g.err;
  z.active = active;
  TcStepArgs st{};
  st.C = C;
  st.D = D;
  st.ld = g.ld;
  st.K = g.npad;
  st.ncols = D;
  st.kc_split = kc_split;
  st.part = g.part;
  st.da = da;
  st.err = g.err;
  st.active = active;
  k_gauss_tc_step<kEpiLrResid, 64, 2><<<dim3(mt, g.nrt), kThreads, Tile<64, 2>::kSmem, s>>>(
      g.mThi[0], g.mTlo[0], g.mXhi, g.mXlo, z);
  launch_tile<kEpiStore>(g.bng, dim3(mt, g.ndt, S), g.mRhi, g.mRlo, g.mXThi, g.mXTlo, st, s);
  count_launch(2);
  *splits = S;
  return cudaGetLastError();
}

}  // namespace hmc
