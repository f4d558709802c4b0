// Bayesian logistic regression on the tcgen05 tensor cores: each leapfrog
// gradient is two chain-batched products back to back (Section 2.1's batched
// target evaluation of a "list of vectors"), 3xTF32 with float32 accumulation:
//   Z = Theta X^T          (M = 256 chains, N = 128 data rows, K = D)
//   R = y - sigmoid(Z)     (epilogue, straight back into tensor memory)
//   G += R X               (M = 256 chains, N = D, K = 128 data rows; A = R
//                           read from tensor memory, B = the transposed data)
// on CTA pairs (tcgen05 cta_group::2): each CTA holds 128 of the chains (its
// rows of Theta, Z, R and G) and loads half of every data tile -- 64 rows of
// X for Z, half of the dims of X^T for G -- so each SM reads half the data
// and issues half the MMAs of a one-CTA tile, and the pair exchanges nothing
// but barrier arrivals.  With one CTA per 128 chains, the first product read
// 8 KB of shared memory per MMA and issued at 53 ns instead of 33.
// Z is double-buffered in tensor memory and R's head is written over the Z it
// came from, so the tensor pipe computes Z of the next tile while the
// epilogue turns this tile's Z into R; R's remainder has one buffer, which
// the epilogue refills once the previous tile's G products are done.
// One CTA pair per (256-chain group, range of data rows); the data tiles
// stream by TMA through a ring of stages and every tile serves all 256
// chains; Z and R never reach HBM.  Per-range partial gradients and log-likelihoods are
// summed in a fixed order by k_lr_update, which also applies the leapfrog
// update.  A transition is: begin (momentum, half kick, drift), L x (grad,
// update), accept.  For D <= 128 (tensor memory holds Z, R head / remainder
// and G at once); the workspace's rows are padded to a multiple of 4 floats
// (zeros), so any such D runs here.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

constexpr int kM = 128;                     // chains per CTA
constexpr int kPairM = 2 * kM;              // chains per CTA pair (MMA M)
constexpr int kRowsPerTile = 128;           // data rows per tile
constexpr int kMaxD = 128;
// warp 0 TMA, warp 1 MMA, then kEpiGroups x 4 epilogue warps: a lane
// quarter's warps split the tile's 128 columns into kEpiGroups groups
constexpr int kEpiGroups = 4;
constexpr int kEpiWarps = 4 * kEpiGroups;
constexpr int kGroupCols = 128 / kEpiGroups;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTile = 128 * 128;       // 128 x 32 floats
constexpr uint32_t kHalfTile = 64 * 128;    // 64 x 32 floats: a CTA's half of a data chunk
constexpr uint32_t kStage = 2 * kHalfTile;  // head + remainder
constexpr int kStages = 6;
constexpr uint32_t kThetaBytes = 2 * 4 * kTile;   // 4 K-chunks, head + remainder
// Z / R head of even tiles at 0, of odd tiles at 128; R remainder; G
constexpr uint32_t kColZR = 0, kColRlo = 256, kColG = 384;
constexpr uint32_t kTmemCols = 512;
constexpr size_t kSmem = kThetaBytes + kStages * kStage + 1024 + 256;
static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(kEpiGroups * 128 * 4 <= kStage, "log-likelihood partials reuse stage 0");
static_assert(8 * (2 * kStages + 5) + 16 <= 256, "barriers");

struct LrTcArgs {
  int C, D, N, ntiles, tiles_per_split, nsplit, dpad;
  int ld;                // row length of the workspace arrays (D rounded up to 4)
  int need_lp;           // log-likelihood partials too (last leapfrog step only)
  const float* y;        // [Npad]
  float* Gpart;          // [nsplit x C x D]
  float* lp_part;        // [nsplit x C]
  int* err;
  const uint8_t* active; // null, or per-chain flags: a pair whose 256 chains have none set is skipped
};

__global__ void __launch_bounds__(kThreads, 1)
k_lr_grad(const __grid_constant__ CUtensorMap mThi, const __grid_constant__ CUtensorMap mTlo,
          const __grid_constant__ CUtensorMap mXhi, const __grid_constant__ CUtensorMap mXlo,
          const __grid_constant__ CUtensorMap mXThi, const __grid_constant__ CUtensorMap mXTlo,
          LrTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* Th = smem;                                   // [4 chunks][hi, lo] 16 KB each
  uint8_t* St = smem + kThetaBytes;                     // [kStages][hi, lo] 8 KB each
  uint64_t* full = reinterpret_cast<uint64_t*>(St + kStages * kStage);   // leader's count
  uint64_t* empty = full + kStages;
  uint64_t* th_full = empty + kStages;    // leader: both CTAs' positions loaded
  uint64_t* z_full = th_full + 1;         // [2]: Z of the tile in buffer b is complete
  uint64_t* r_ready = z_full + 2;         // leader: both CTAs' R written
  uint64_t* g_done = r_ready + 1;         // G of a tile is complete (R remainder free)
  uint64_t* g_full = g_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(g_full + 1);
  // [kEpiGroups][128] log-likelihood partials: written after the last MMA,
  // when the data stages are no longer read
  float* lpred = reinterpret_cast<float*>(St);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (a.active) {
    // NUTS: both CTAs of the pair read the same 256 flags and skip together,
    // before anything the pair shares
    const int r = threadIdx.x;
    const int m = (blockIdx.x >> 1) * kPairM + r;
    const bool mine = r < kPairM && m < a.C && a.active[m] != 0;
    if (!__syncthreads_or(mine)) return;
  }
  const uint32_t rank = ptx::cluster_rank();             // 0: leader, 1: peer
  const int m0 = (blockIdx.x >> 1) * kPairM + static_cast<int>(rank) * kM;   // this CTA's chains
  const int split = blockIdx.y;
  const int t_begin = split * a.tiles_per_split;
  const int t_end = min(a.ntiles, t_begin + a.tiles_per_split);
  const int ntile = max(0, t_end - t_begin);
  const int nk = (a.D + 31) >> 5;
  constexpr uint16_t kPairMask = 0x3;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(th_full, 1);
    ptx::mbar_init(&z_full[0], 1);
    ptx::mbar_init(&z_full[1], 1);
    ptx::mbar_init(r_ready, 2 * kEpiWarps);   // one arrival per epilogue warp of the pair
    ptx::mbar_init(g_done, 1);
    ptx::mbar_init(g_full, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc_pair(tmem_slot, kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();      // both CTAs' barriers and tensor memory exist
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0 && ntile > 0) {
      // ---- producer (both CTAs): this CTA's chains' positions once, then per
      // tile its half of the data (rows for Z, dims for G), completing on the
      // leader's barriers
      const uint32_t th_bar = ptx::mapa(ptx::smem_u32(th_full), 0);
      if (rank == 0) ptx::mbar_arrive_expect_tx(th_full, 2u * 2u * nk * kTile);
      for (int kc = 0; kc < nk; ++kc) {
        ptx::tma_load_2d_to_bar(Th + (2 * kc) * kTile, &mThi, th_bar, kc * 32, m0);
        ptx::tma_load_2d_to_bar(Th + (2 * kc + 1) * kTile, &mTlo, th_bar, kc * 32, m0);
      }
      int it = 0;
      auto stage = [&](const CUtensorMap* mh, const CUtensorMap* ml, int c0, int c1) {
        const int s = it % kStages, round = it / kStages;
        ++it;
        if (it > kStages && !ptx::mbar_wait(&empty[s], (round - 1) & 1)) {
          atomicCAS(a.err, 0, 11);
          ok = false;
          return;
        }
        uint8_t* st = St + s * kStage;
        if (rank == 0) ptx::mbar_arrive_expect_tx(&full[s], 2u * kStage);
        const uint32_t bar = ptx::mapa(ptx::smem_u32(&full[s]), 0);
        ptx::tma_load_2d_to_bar(st, mh, bar, c0, c1);
        ptx::tma_load_2d_to_bar(st + kHalfTile, ml, bar, c0, c1);
      };
      // stages in the order the issuer consumes them: Z(0), then per tile
      // ti: Z(ti + 1), G(ti)
      const int dhalf = a.dpad / 2;
      auto load_z = [&](int ti) {
        const int row0 = (t_begin + ti) * kRowsPerTile + static_cast<int>(rank) * (kRowsPerTile / 2);
        for (int part = 0; part < nk && ok; ++part) stage(&mXhi, &mXlo, part * 32, row0);
      };
      auto load_g = [&](int ti) {
        const int row0 = (t_begin + ti) * kRowsPerTile;
        for (int kr = 0; kr < 4 && ok; ++kr)
          stage(&mXThi, &mXTlo, row0 + kr * 32, static_cast<int>(rank) * dhalf);
      };
      load_z(0);
      for (int ti = 0; ti < ntile && ok; ++ti) {
        if (ti + 1 < ntile) load_z(ti + 1);
        load_g(ti);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && ntile > 0 && rank == 0) {
      // ---- MMA issuer (leader): M = 256 chains across the pair
      const uint32_t idesc1 = ptx::idesc_tf32(kPairM, kRowsPerTile);
      const uint32_t idesc2 = ptx::idesc_tf32(kPairM, a.dpad);
      if (!ptx::mbar_wait(th_full, 0)) {
        atomicCAS(a.err, 0, 12);
        ok = false;
      }
      ptx::tc_fence_after();
      int it = 0;
      // Z = Theta X^T into buffer ti % 2 (N = the tile's 128 rows, 64 per CTA)
      auto mma_z = [&](int ti) {
        const uint32_t zcol = tmem + kColZR + 128u * static_cast<uint32_t>(ti & 1);
        for (int kc = 0; kc < nk && ok; ++kc, ++it) {
          const int s = it % kStages;
          if (!ptx::mbar_wait(&full[s], (it / kStages) & 1)) {
            atomicCAS(a.err, 0, 13);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t thi = ptx::smem_u32(Th + (2 * kc) * kTile);
          const uint32_t tlo = ptx::smem_u32(Th + (2 * kc + 1) * kTile);
          const uint32_t xhi = ptx::smem_u32(St + s * kStage);
          const uint32_t xlo = xhi + kHalfTile;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t dth = ptx::sw128_kmajor_desc(thi + 32 * j);
            const uint64_t dtl = ptx::sw128_kmajor_desc(tlo + 32 * j);
            const uint64_t dxh = ptx::sw128_kmajor_desc(xhi + 32 * j);
            const uint64_t dxl = ptx::sw128_kmajor_desc(xlo + 32 * j);
            ptx::mma_tf32_pair(zcol, dtl, dxh, idesc1, (kc | j) != 0 ? 1u : 0u);
            ptx::mma_tf32_pair(zcol, dth, dxl, idesc1, 1u);
            ptx::mma_tf32_pair(zcol, dth, dxh, idesc1, 1u);
          }
          ptx::mma_commit_pair(&empty[s], kPairMask);
        }
        if (ok) ptx::mma_commit_pair(&z_full[ti & 1], kPairMask);
      };
      // G += R X   (A = R from each CTA's tensor memory, N = dims, half per CTA)
      auto mma_g = [&](int ti) {
        if (!ptx::mbar_wait_cluster(r_ready, ti & 1)) {
          atomicCAS(a.err, 0, 14);
          ok = false;
          return;
        }
        ptx::tc_fence_after();
        const uint32_t rhi = tmem + kColZR + 128u * static_cast<uint32_t>(ti & 1);
        for (int kr = 0; kr < 4 && ok; ++kr, ++it) {
          const int s = it % kStages;
          if (!ptx::mbar_wait(&full[s], (it / kStages) & 1)) {
            atomicCAS(a.err, 0, 15);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t bhi = ptx::smem_u32(St + s * kStage);
          const uint32_t blo = bhi + kHalfTile;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t dbh = ptx::sw128_kmajor_desc(bhi + 32 * j);
            const uint64_t dbl = ptx::sw128_kmajor_desc(blo + 32 * j);
            const uint32_t k = static_cast<uint32_t>(kr * 32 + 8 * j);
            ptx::mma_tf32_pair_tmem_a(tmem + kColG, tmem + kColRlo + k, dbh, idesc2,
                                      (ti | kr | j) != 0 ? 1u : 0u);
            ptx::mma_tf32_pair_tmem_a(tmem + kColG, rhi + k, dbl, idesc2, 1u);
            ptx::mma_tf32_pair_tmem_a(tmem + kColG, rhi + k, dbh, idesc2, 1u);
          }
          ptx::mma_commit_pair(&empty[s], kPairMask);
        }
        if (ok) ptx::mma_commit_pair(g_done, kPairMask);
      };
      // MMAs execute in issue order: Z(ti + 1) overwrites the buffer G(ti - 1)
      // read only after G(ti - 1)
      mma_z(0);
      for (int ti = 0; ti < ntile && ok; ++ti) {
        if (ti + 1 < ntile) mma_z(ti + 1);
        mma_g(ti);
      }
      ptx::mma_commit_pair(g_full, kPairMask);
    }
  } else {
    // ---- epilogue (both CTAs): thread = chain row (TMEM lane), one group of columns
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int group = ew >> 2;
    const int r = quarter * 32 + lane;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    const uint32_t r_ready_leader = ptx::mapa(ptx::smem_u32(r_ready), 0);
    float lp_acc = 0.f;
    const bool need_lp = a.need_lp != 0;
    for (int ti = 0; ti < ntile; ++ti) {
      const int row0 = (t_begin + ti) * kRowsPerTile;
      const uint32_t zr = tmem + lane_base + kColZR + 128u * static_cast<uint32_t>(ti & 1);
      if (!ptx::mbar_wait(&z_full[ti & 1], (ti >> 1) & 1)) {
        atomicCAS(a.err, 0, 16);
        ok = false;
      }
      ptx::tc_fence_after();
      // R's head goes over Z block by block; its remainder waits in
      // registers until the previous tile's G products release the buffer
      float rl[kGroupCols];
#pragma unroll
      for (int cb = 0; cb < kGroupCols / 16; ++cb) {
        const uint32_t col = static_cast<uint32_t>(kGroupCols * group + 16 * cb);
        float zv[16], rh[16];
        ptx::tmem_ld16(zr + col, zv);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int n = row0 + static_cast<int>(col) + k;
          float res = 0.f;
          if (n < a.N) {              // warp-uniform: a warp's lanes are chains
            const float yv = a.y[n];
            res = residual_f(yv, zv[k]);
            if (need_lp) lp_acc += loglik_f(yv, zv[k]);
          }
          split_tf32(res, rh[k], rl[16 * cb + k]);
        }
        ptx::tmem_st16(zr + col, rh);
      }
      if (ti > 0) {
        if (!ptx::mbar_wait(g_done, (ti - 1) & 1)) {
          atomicCAS(a.err, 0, 18);
          ok = false;
        }
        ptx::tc_fence_after();
      }
#pragma unroll
      for (int cb = 0; cb < kGroupCols / 16; ++cb)
        ptx::tmem_st16(tmem + lane_base + kColRlo + kGroupCols * group + 16 * cb, rl + 16 * cb);
      ptx::tmem_wait_st();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          ptx::mbar_arrive_local(r_ready);
        else
          ptx::mbar_arrive_cluster(r_ready_leader);
      }
    }
    // partial gradient and log-likelihood of this row range
    const int chain = m0 + r;
    if (ntile > 0) {
      if (!ptx::mbar_wait(g_full, 0)) {
        atomicCAS(a.err, 0, 17);
        ok = false;
      }
      ptx::tc_fence_after();
    }
    float* gout = a.Gpart + (static_cast<int64_t>(split) * a.C + chain) * a.ld;
#pragma unroll 1
    for (int cb = 0; cb < kGroupCols / 16; ++cb) {
      const int d0 = kGroupCols * group + 16 * cb;
      if (d0 >= a.dpad) break;                    // warp-uniform
      float gv[16];
      if (ntile > 0) {
        ptx::tmem_ld16(tmem + lane_base + kColG + static_cast<uint32_t>(d0), gv);
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) gv[k] = 0.f;
      }
      if (ok && chain < a.C)
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (d0 + k < a.ld) gout[d0 + k] = gv[k];    // (zero past D: X's padding)
    }
    lpred[group * 128 + r] = lp_acc;
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp >= 2 && warp < 6) {
    const int r = (warp & 3) * 32 + lane;
    const int chain = m0 + r;
    if (ok && chain < a.C) {
      float lp = 0.f;
#pragma unroll
      for (int g = 0; g < kEpiGroups; ++g) lp += lpred[g * 128 + r];
      a.lp_part[static_cast<int64_t>(split) * a.C + chain] = lp;
    }
  }
  ptx::cluster_sync();      // the peer no longer needs this CTA's tensor memory
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, kTmemCols);
  }
}

constexpr int kWarpsPerBlock = 8;

struct LrStepArgs {
  StepArgs s;
  int ld;           // row length of the workspace arrays below (D rounded up to 4; zero past D)
  float* thi;       // [C x ld] positions, tf32 head / remainder (A operand)
  float* tlo;
  float* p;         // [C x ld] momenta
  float* gL;        // [C x ld] gradient at the end of the trajectory
  float* lpL;       // [C]
  float* h0;        // [C]
  const float* Gpart;
  const float* lp_part;
  int nsplit;
  int last;         // update kernel: final leapfrog step
};

// p0 ~ N(0, I); H0; half kick with the cached gradient; first drift
__global__ void k_lr_begin(LrStepArgs b) {
  const StepArgs& a = b.s;
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.C) return;
  const int D = a.D;
  const int64_t row = static_cast<int64_t>(c) * D, wrow = static_cast<int64_t>(c) * b.ld;
  const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
  const float eps = a.da->eps;
  float kin = 0.f;
  for (int d = lane; d < D; d += 32) {
    const float z = momentum1(a.seed, static_cast<uint32_t>(d), chain, a.t);
    kin = fmaf(z, z, kin);
    const float p = fmaf(0.5f * eps, a.g[row + d], z);
    b.p[wrow + d] = p;
    float hi, lo;
    split_tf32(fmaf(eps, p, a.x[row + d]), hi, lo);
    b.thi[wrow + d] = hi;
    b.tlo[wrow + d] = lo;
  }
  kin = warp_sum(kin);
  if (lane == 0) b.h0[c] = -a.lp[c] + 0.5f * kin;
}

// gradient and log p from the range partials (fixed order) and the prior;
// leapfrog update (merged kicks + drift), or the final half kick.  One warp
// per chain, four dims per lane (float4: every buffer here is the library's
// own, 16-byte aligned, with rows of ld = D rounded up to 4), so that a
// lane's loads of all range partials are in flight together.
__global__ void k_lr_update(LrStepArgs b) {
  const StepArgs& a = b.s;
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.C) return;
  const int D4 = b.ld >> 2;           // (the padding stays zero: X's padding columns are zero)
  const int64_t row4 = static_cast<int64_t>(c) * D4;
  const int64_t split4 = static_cast<int64_t>(a.C) * D4;
  const float eps = a.da->eps;
  const float4* thi = reinterpret_cast<const float4*>(b.thi);
  const float4* tlo = reinterpret_cast<const float4*>(b.tlo);
  const float4* Gp = reinterpret_cast<const float4*>(b.Gpart);
  float4* p4 = reinterpret_cast<float4*>(b.p);
  float sq = 0.f;
  for (int j = lane; j < D4; j += 32) {
    const int64_t e = row4 + j;
    const float4 h = thi[e], l = tlo[e];
    const float th[4] = {h.x + l.x, h.y + l.y, h.z + l.z, h.w + l.w};
    float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int s = 0; s < b.nsplit; ++s) {
      const float4 v = Gp[s * split4 + e];
      g[0] += v.x; g[1] += v.y; g[2] += v.z; g[3] += v.w;
    }
    const float4 pv = p4[e];
    const float pin[4] = {pv.x, pv.y, pv.z, pv.w};
    float pout[4], hi[4], lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g[k] -= th[k];
      sq = fmaf(th[k], th[k], sq);
      if (!b.last) {
        pout[k] = fmaf(eps, g[k], pin[k]);
        split_tf32(fmaf(eps, pout[k], th[k]), hi[k], lo[k]);
      } else {
        pout[k] = fmaf(0.5f * eps, g[k], pin[k]);
      }
    }
    p4[e] = make_float4(pout[0], pout[1], pout[2], pout[3]);
    if (!b.last) {
      reinterpret_cast<float4*>(b.thi)[e] = make_float4(hi[0], hi[1], hi[2], hi[3]);
      reinterpret_cast<float4*>(b.tlo)[e] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    } else {
      reinterpret_cast<float4*>(b.gL)[e] = make_float4(g[0], g[1], g[2], g[3]);
    }
  }
  if (b.last) {
    sq = warp_sum(sq);
    if (lane == 0) {
      float lp = 0.f;
      for (int s = 0; s < b.nsplit; ++s) lp += b.lp_part[static_cast<int64_t>(s) * a.C + c];
      b.lpL[c] = lp - 0.5f * sq;
    }
  }
}

// H_L, Metropolis-Hastings select, traces, dual averaging
__global__ void k_lr_accept(LrStepArgs b) {
  const StepArgs& a = b.s;
  const int c = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool has_chain = c < a.C;
  float prob = 0.f;
  if (has_chain) {
    const int D = a.D;
    const int64_t row = static_cast<int64_t>(c) * D, wrow = static_cast<int64_t>(c) * b.ld;
    const uint32_t chain = static_cast<uint32_t>(c) + a.chain_offset;
    float kin = 0.f;
    for (int d = lane; d < D; d += 32) kin = fmaf(b.p[wrow + d], b.p[wrow + d], kin);
    kin = 0.5f * warp_sum(kin);
    const float lp1 = b.lpL[c];
    float la = b.h0[c] - (-lp1 + kin);
    if (!isfinite(la)) la = -INFINITY;
    int acc = 0;
    if (lane == 0) acc = accept_log_uniform(a.seed, chain, a.t) < la;
    acc = __shfl_sync(0xffffffffu, acc, 0);
    for (int d = lane; d < D; d += 32) {
      const int64_t e = row + d, w = wrow + d;
      if (acc) {
        a.x[e] = b.thi[w] + b.tlo[w];
        a.g[e] = b.gL[w];
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

// X -> head / remainder [Npad x ld], and the transposed copy [ld x Npad];
// rows >= N and columns >= D zero (ld >= D: the padded row length)
__global__ void k_lr_prepare(int N, int Npad, int D, int ld, const float* __restrict__ X,
                             const float* __restrict__ y, float* __restrict__ Xhi,
                             float* __restrict__ Xlo, float* __restrict__ XThi,
                             float* __restrict__ XTlo, float* __restrict__ ypad) {
  const int64_t total = static_cast<int64_t>(Npad) * ld;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int n = static_cast<int>(i / ld), d = static_cast<int>(i % ld);
    const float v = n < N && d < D ? X[static_cast<int64_t>(n) * D + d] : 0.f;
    float hi, lo;
    split_tf32(v, hi, lo);
    Xhi[i] = hi;
    Xlo[i] = lo;
    XThi[static_cast<int64_t>(d) * Npad + n] = hi;
    XTlo[static_cast<int64_t>(d) * Npad + n] = lo;
    if (d == 0) ypad[n] = n < N ? y[n] : 0.f;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode() {
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

bool map2d(CUtensorMap* m, const float* base, int64_t rows, int64_t cols, unsigned box_rows) {
  auto fn = encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * sizeof(float)};
  cuuint32_t box[2] = {32u, box_rows};
  cuuint32_t es[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t a1k(size_t b) { return (b + 1023) & ~static_cast<size_t>(1023); }

// row length of the workspace arrays: the dim rounded up to 4 floats (TMA
// strides are multiples of 16 bytes); the padding columns hold zeros
inline int lr_ld(int dim) { return (dim + 3) / 4 * 4; }

struct Plan {
  int npad, ntiles, groups, nsplit, tps, dpad;
};

Plan plan(const hmc_target& t, int64_t C) {
  Plan p{};
  p.ntiles = static_cast<int>((t.n_data + kRowsPerTile - 1) / kRowsPerTile);
  p.npad = p.ntiles * kRowsPerTile;
  p.groups = static_cast<int>((C + kPairM - 1) / kPairM);   // CTA pairs
  int ns = std::max(1, 76 / p.groups);
  ns = std::min(ns, p.ntiles);
  p.tps = (p.ntiles + ns - 1) / ns;
  p.nsplit = (p.ntiles + p.tps - 1) / p.tps;
  p.dpad = (t.dim + 15) / 16 * 16;
  return p;
}

}  // namespace

cudaError_t launch_lr_prepare(int N, int Npad, int D, int ld, const float* X, const float* y, float* Xhi,
                              float* Xlo, float* XThi, float* XTlo, float* ypad, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(Npad) * ld;
  k_lr_prepare<<<static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 152 * 16)), 256, 0, s>>>(
      N, Npad, D, ld, X, y, Xhi, Xlo, XThi, XTlo, ypad);
  count_launch();
  return cudaGetLastError();
}

bool logreg_tc_supported(const hmc_target& t) {
  return t.id == HMC_T_LOGREG && t.dim <= kMaxD && encode() != nullptr;
}

size_t logreg_tc_workspace_bytes(const hmc_target& t, int64_t C) {
  const Plan p = plan(t, C);
  const size_t ld = static_cast<size_t>(lr_ld(t.dim));
  const size_t CD = static_cast<size_t>(C) * ld, ND = static_cast<size_t>(p.npad) * ld;
  return 4 * a1k(ND * 4) + a1k(p.npad * 4) + 4 * a1k(CD * 4) + a1k(C * 4) * 2 +
         a1k(static_cast<size_t>(p.nsplit) * CD * 4) + a1k(static_cast<size_t>(p.nsplit) * C * 4);
}

cudaError_t logreg_tc_setup(LogregTc* tc, const hmc_target& t, int64_t C, void* ws, cudaStream_t s) {
  const Plan p = plan(t, C);
  tc->npad = p.npad;
  tc->ntiles = p.ntiles;
  tc->nsplit = p.nsplit;
  tc->tps = p.tps;
  tc->groups = p.groups;
  tc->dpad = p.dpad;
  tc->n_data = static_cast<int>(t.n_data);
  tc->ld = lr_ld(t.dim);
  const size_t CD = static_cast<size_t>(C) * tc->ld, ND = static_cast<size_t>(p.npad) * tc->ld;
  char* w = static_cast<char*>(ws);
  auto take = [&](size_t b) { char* q = w; w += a1k(b); return reinterpret_cast<float*>(q); };
  tc->Xhi = take(ND * 4);
  tc->Xlo = take(ND * 4);
  tc->XThi = take(ND * 4);
  tc->XTlo = take(ND * 4);
  tc->ypad = take(p.npad * 4);
  tc->thi = take(CD * 4);
  tc->tlo = take(CD * 4);
  tc->p = take(CD * 4);
  tc->gL = take(CD * 4);
  tc->lpL = take(C * 4);
  tc->h0 = take(C * 4);
  tc->Gpart = take(static_cast<size_t>(p.nsplit) * CD * 4);
  tc->lp_part = take(static_cast<size_t>(p.nsplit) * C * 4);
  const int ld = tc->ld;
  const bool ok = map2d(&tc->mThi, tc->thi, C, ld, 128) && map2d(&tc->mTlo, tc->tlo, C, ld, 128) &&
                  map2d(&tc->mXhi, tc->Xhi, p.npad, ld, 64) &&
                  map2d(&tc->mXlo, tc->Xlo, p.npad, ld, 64) &&
                  map2d(&tc->mXThi, tc->XThi, ld, p.npad, 64) &&
                  map2d(&tc->mXTlo, tc->XTlo, ld, p.npad, 64);
  if (!ok) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_lr_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kSmem));
  if (e != cudaSuccess) return e;
  const int64_t total = static_cast<int64_t>(p.npad) * ld;
  k_lr_prepare<<<static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 152 * 16)), 256, 0, s>>>(
      static_cast<int>(t.n_data), p.npad, t.dim, ld, t.X, t.y, tc->Xhi, tc->Xlo, tc->XThi, tc->XTlo,
      tc->ypad);
  count_launch();
  // the positions' and momenta's padding columns (ld > D) are read but never
  // written: zero once (thi, tlo, p, gL are contiguous)
  e = cudaMemsetAsync(tc->thi, 0, reinterpret_cast<char*>(tc->gL) + a1k(CD * 4) - reinterpret_cast<char*>(tc->thi), s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_logreg_tc_grad(LogregTc& tc, int C, int D, const uint8_t* active, int* err, cudaStream_t s) {
  LrTcArgs g{};
  g.C = C;
  g.D = D;
  g.ntiles = tc.ntiles;
  g.tiles_per_split = tc.tps;
  g.nsplit = tc.nsplit;
  g.dpad = tc.dpad;
  g.y = tc.ypad;
  g.Gpart = tc.Gpart;
  g.lp_part = tc.lp_part;
  g.err = err;
  g.N = tc.n_data;
  g.need_lp = 1;
  g.active = active;
  g.ld = tc.ld;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * tc.groups, tc.nsplit);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_lr_grad, tc.mThi, tc.mTlo, tc.mXhi, tc.mXlo, tc.mXThi,
                                           tc.mXTlo, g);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_logreg_tc_transition(const StepArgs& a, LogregTc& tc, int* err, cudaStream_t s,
                                        KernelTimer* timer) {
  LrStepArgs b{};
  b.s = a;
  b.ld = tc.ld;
  b.thi = tc.thi;
  b.tlo = tc.tlo;
  b.p = tc.p;
  b.gL = tc.gL;
  b.lpL = tc.lpL;
  b.h0 = tc.h0;
  b.Gpart = tc.Gpart;
  b.lp_part = tc.lp_part;
  b.nsplit = tc.nsplit;
  const unsigned nb = static_cast<unsigned>((a.C + kWarpsPerBlock - 1) / kWarpsPerBlock);
  k_lr_begin<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
  count_launch();
  LrTcArgs g{};
  g.C = a.C;
  g.D = a.D;
  g.ntiles = tc.ntiles;
  g.tiles_per_split = tc.tps;
  g.nsplit = tc.nsplit;
  g.dpad = tc.dpad;
  g.y = tc.ypad;
  g.Gpart = tc.Gpart;
  g.lp_part = tc.lp_part;
  g.err = err;
  g.N = tc.n_data;
  g.ld = tc.ld;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * tc.groups, tc.nsplit);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (int l = 1; l <= a.L; ++l) {
    g.need_lp = l == a.L;
    if (timer) timer->begin(s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_lr_grad, tc.mThi, tc.mTlo, tc.mXhi, tc.mXlo, tc.mXThi,
                                       tc.mXTlo, g);
    if (timer) timer->end(s);
    if (e != cudaSuccess) return e;
    b.last = l == a.L;
    k_lr_update<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
    count_launch(2);
  }
  k_lr_accept<<<nb, 32 * kWarpsPerBlock, 0, s>>>(b);
  count_launch();
  return cudaGetLastError();
}

}  // namespace hmc
