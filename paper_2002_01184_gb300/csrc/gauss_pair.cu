// One launch per HMC transition for the dense Gaussian target (dim <= 256) on
// CTA pairs (tcgen05 cta_group::2).  A pair owns 64 chains for the whole
// transition (Section 2.1): each leapfrog gradient G^T = P X^T is one stream
// of M = 256 (all output dims), N = 64 (the pair's chains), K = 8 MMAs issued
// by the pair's leader.
//   * A (P head / remainder, 3xTF32) is resident for the whole launch: each
//     CTA's 128 rows of P, K-chunks 0-6 (dims 0-223) in its tensor memory and
//     chunk 7 (dims 224-255) in shared memory.  The MMAs then read only the
//     positions from shared memory: at 64 chains an MMA that also read A from
//     shared memory would be bound by shared-memory bandwidth, not by the
//     tensor pipe.
//   * B (positions, head / remainder tiles, 128-byte-swizzled K-major): each
//     CTA holds 32 of the 64 chains.
//   * Accumulators: each CTA's tensor memory holds its 128 output dims for
//     all 64 chains.
//   * Epilogue (warps 2-9 of both CTAs): one output dim per thread, 32 chains
//     per thread; momenta and positions stay in registers.  The next
//     positions of this CTA's own chains go straight into its tile; those of
//     the peer's chains are staged locally (in the destination's layout) and
//     each staging warp pushes its K-chunk (head and remainder, 4 KB each) to
//     the peer by bulk DSMEM copy, completing on the peer's tile barrier --
//     element-wise remote stores stalled every warp's shared-memory traffic.
//   * Readiness is tracked per half of K: in each CTA's tile the K-chunks of
//     its own dims are written locally (own_full, which every epilogue thread
//     joins once it has read the accumulators) and the other four arrive by
//     copy (in_full).
//     The peer forwards both completions to the leader.  The issuer starts
//     on K-chunks 4-7, whose leader half arrives by copy straight onto the
//     leader's barrier, and reaches K-chunks 0-3, whose peer half needs the
//     copy plus the forward, a quarter-step of MMAs later.
// H_L, the Metropolis-Hastings decision and the dual-averaging partial are
// formed by the leader from both CTAs' partial sums.
#include <cuda.h>

#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

constexpr int kMaxDim = 256;
constexpr int kChunks = kMaxDim / 32;             // K-chunks of 32 dims
constexpr int kTmemChunks = 7;                    // P chunks held in tensor memory
constexpr int kThreads = 320;
constexpr int kPairChains = 64;                   // MMA N
constexpr int kHalf = 32;                         // chains per CTA (B rows)
constexpr uint32_t kBChunk = kHalf * 128;         // 32 rows x 128 B
constexpr uint32_t kBBytes = kChunks * kBChunk;   // head or remainder tile
constexpr uint32_t kAHalf = 128 * 128;            // 128 rows x 32 floats
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColAcc = 0;                   // accumulators: 64 columns
constexpr uint32_t kColP = 64;                    // chunk kc: head at kColP + 64 kc, remainder + 32
constexpr uint32_t kStageHalf = 4 * kBChunk;      // 4 K-chunks (this CTA's 128 dims) x 32 chains
constexpr uint32_t kStageBytes = 2 * kStageHalf;  // head + remainder: one bulk copy each
// barriers, tmem slot, red [2][4][64], red_pair [2][64], peer_in [2][64],
// acc_flag [64], prob_s [64]
constexpr uint32_t kSmall = 8 * 6 + 8 + (2 * 4 * 64 + 2 * 64 + 2 * 64 + 64 + 64) * 4;
constexpr size_t kSmemUsed = 2 * kBBytes + 2 * kAHalf + 2 * kStageBytes + kSmall + 1024;
// Above half of an SM's shared memory, so that one CTA runs per SM: a CTA
// allocates all 512 tensor-memory columns and must never queue in
// tcgen05.alloc behind another CTA of the launch.
constexpr size_t kSmem = kSmemUsed > 120 * 1024 ? kSmemUsed : 120 * 1024;

struct PairArgs {
  StepArgs s;
  int* err;
  const float* p0;      // [C x D]
  const float* kin0;    // [C]
  const float* Ptm;     // P chunks 0-6 in tensor-memory fill order (k_tmem_image)
};

// Index of element e of float4 j of lane `lane` in the tensor-memory image:
// rank, K-chunk kc (0-6), head / remainder hl, 16-column half q16, lane
// quarter q.  A warp's j-th float4 load of a 16-column block is 512
// contiguous bytes.
__host__ __device__ constexpr int image_index(int rank, int kc, int hl, int q16, int q, int j, int lane) {
  return (((((rank * kTmemChunks + kc) * 2 + hl) * 2 + q16) * 4 + q) * 4 + j) * 128 + lane * 4;
}

__global__ void k_tmem_image(const float* __restrict__ Phi, const float* __restrict__ Plo, int D,
                             float* __restrict__ image) {
  constexpr int n = 2 * kTmemChunks * 2 * 2 * 4 * 4 * 32;   // float4 slots
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int r = v;
    const int lane = r % 32; r /= 32;
    const int j = r % 4; r /= 4;
    const int q = r % 4; r /= 4;
    const int q16 = r % 2; r /= 2;
    const int hl = r % 2; r /= 2;
    const int kc = r % kTmemChunks;
    const int rank = r / kTmemChunks;
    const int row = rank * 128 + q * 32 + lane;
    const int col = kc * 32 + q16 * 16 + j * 4;
    const float* src = hl == 0 ? Phi : Plo;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < D && col < D)            // D % 4 == 0: all four in or out
      val = *reinterpret_cast<const float4*>(src + static_cast<int64_t>(row) * D + col);
    *reinterpret_cast<float4*>(image + image_index(rank, kc, hl, q16, q, j, lane)) = val;
  }
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence_cta() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
k_gauss_pair(const __grid_constant__ CUtensorMap mPhi, const __grid_constant__ CUtensorMap mPlo,
             PairArgs fa) {
  const StepArgs& a = fa.s;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* Bhi = smem;
  uint8_t* Blo = smem + kBBytes;
  uint8_t* A7 = smem + 2 * kBBytes;                        // P chunk 7: head, remainder
  uint8_t* Stg = A7 + 2 * kAHalf;                          // [2 buffers][head, remainder]
  uint64_t* a7_full = reinterpret_cast<uint64_t*>(Stg + 2 * kStageBytes);
  uint64_t* acc_full = a7_full + 1;
  uint64_t* own_full = acc_full + 1;      // all epilogue threads: accumulators read, own K-chunks written
  uint64_t* in_full = own_full + 1;       // this CTA's tile: the peer's K-chunks copied in
  uint64_t* fwd_own = in_full + 1;        // leader: the peer's own_full, forwarded
  uint64_t* fwd_in = fwd_own + 1;         // leader: the peer's in_full, forwarded
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fwd_in + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 2);   // [2][4 quarters][64 chains]
  float* red_pair = red + 2 * 4 * 64;                     // [2][64] this CTA's sums
  float* peer_in = red_pair + 2 * 64;                     // [2][64] the peer's sums (leader)
  int* acc_flag = reinterpret_cast<int*>(peer_in + 2 * 64);   // [64]
  float* prob_s = reinterpret_cast<float*>(acc_flag + 64);    // [64]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_rank();              // 0: leader, 1: peer
  const int C = a.C, D = a.D, L = a.L;
  const int nk = (D + 31) >> 5;
  const int pair_base = (blockIdx.x >> 1) * kPairChains;
  constexpr uint16_t kPairMask = 0x3;

  if (threadIdx.x == 0) {
    ptx::mbar_init(a7_full, 1);
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(own_full, 256);        // every epilogue thread
    ptx::mbar_init(in_full, 1);           // armed with the copy bytes by one own-chain thread
    ptx::mbar_init(fwd_own, 1);
    ptx::mbar_init(fwd_in, 1);
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mPhi);
    ptx::prefetch_tensormap(&mPlo);
  }
  if (warp == 0) {
    ptx::tmem_alloc_pair(tmem_slot, kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  // B tiles and staging start zeroed: dims >= D are never written
  for (uint32_t i = threadIdx.x; i < 2 * kBBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (uint32_t i = threadIdx.x; i < 2 * kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(Stg)[i] = make_uint4(0u, 0u, 0u, 0u);
  {
    // the begin phase reads x, g and p0 of the pair's chains after the
    // tensor-memory fill: start pulling this CTA's 32 rows of each into L2
    const int c0 = pair_base + static_cast<int>(rank) * kHalf;
    const int rows = max(0, min(kHalf, C - c0));
    const int64_t lines = (static_cast<int64_t>(rows) * D * 4 + 127) / 128;
    const int64_t row0 = static_cast<int64_t>(c0) * D;
    for (int64_t i = threadIdx.x; i < 3 * lines; i += kThreads) {
      const int64_t arr = i / lines, ln = i - arr * lines;
      const float* base = arr == 0 ? a.x : arr == 1 ? a.g : fa.p0;
      const int64_t off = min(ln * 128, static_cast<int64_t>(rows) * D * 4 - 4);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(base + row0) + off));
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();      // both CTAs' barriers and tensor memory exist
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const float eps = a.da->eps;
  const uint32_t peer = 1u - rank;
  bool ok = true;

  // epilogue-thread state (warps 2-9)
  const int ew = warp - 2;
  const int h = ew >> 2;                  // chain half 0 / 1 (= the CTA holding those chains)
  const int quarter = warp & 3;           // tensor-memory lane quarter
  const int d = static_cast<int>(rank) * 128 + quarter * 32 + lane;
  const bool dvalid = warp >= 2 && d < D;
  float p[kHalf], x[kHalf];

  if (warp == 0) {
    if (lane == 0 && nk > kTmemChunks) {
      // ---- P chunk 7 of this CTA's rows, once, completing on the leader's barrier
      if (rank == 0) ptx::mbar_arrive_expect_tx(a7_full, 4 * kAHalf);
      const uint32_t bar = ptx::mapa(ptx::smem_u32(a7_full), 0);
      ptx::tma_load_2d_to_bar(A7, &mPhi, bar, kTmemChunks * 32, static_cast<int>(rank) * 128);
      ptx::tma_load_2d_to_bar(A7 + kAHalf, &mPlo, bar, kTmemChunks * 32, static_cast<int>(rank) * 128);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---- MMA issuer (leader): M = 256 across the pair, N = 64 chains
      constexpr uint32_t idesc = ptx::idesc_tf32(256, kPairChains);
      if (nk > kTmemChunks && !ptx::mbar_wait(a7_full, 0)) {
        atomicCAS(fa.err, 0, 1);
        ok = false;
      }
      // one K-chunk: 4 k-steps x 3 products
      auto chunk_mmas = [&](int kc, bool& first) {
        const uint32_t bhi = ptx::smem_u32(Bhi + kc * kBChunk);
        const uint32_t blo = ptx::smem_u32(Blo + kc * kBChunk);
        if (kc < kTmemChunks) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t dbhi = ptx::sw128_kmajor_desc(bhi + 32 * j);
            const uint64_t dblo = ptx::sw128_kmajor_desc(blo + 32 * j);
            const uint32_t ahi = tmem + kColP + 64 * kc + 8 * j;
            const uint32_t alo = ahi + 32;
            ptx::mma_tf32_pair_tmem_a(tmem + kColAcc, alo, dbhi, idesc, first ? 0u : 1u);
            ptx::mma_tf32_pair_tmem_a(tmem + kColAcc, ahi, dblo, idesc, 1u);
            ptx::mma_tf32_pair_tmem_a(tmem + kColAcc, ahi, dbhi, idesc, 1u);
            first = false;
          }
        } else {
          const uint32_t ahi = ptx::smem_u32(A7);
          const uint32_t alo = ahi + kAHalf;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t dahi = ptx::sw128_kmajor_desc(ahi + 32 * j);
            const uint64_t dalo = ptx::sw128_kmajor_desc(alo + 32 * j);
            const uint64_t dbhi = ptx::sw128_kmajor_desc(bhi + 32 * j);
            const uint64_t dblo = ptx::sw128_kmajor_desc(blo + 32 * j);
            ptx::mma_tf32_pair(tmem + kColAcc, dalo, dbhi, idesc, first ? 0u : 1u);
            ptx::mma_tf32_pair(tmem + kColAcc, dahi, dblo, idesc, 1u);
            ptx::mma_tf32_pair(tmem + kColAcc, dahi, dbhi, idesc, 1u);
            first = false;
          }
        }
      };
      for (int l = 1; l <= L && ok; ++l) {
        const uint32_t ph = (l - 1) & 1;
        bool first = true;
        // K-chunks 4-7: leader half copied in from the peer, peer half local
        // there; own_full and fwd_own also mean both CTAs' epilogues have
        // read the accumulators this step overwrites
        if (!ptx::mbar_wait(own_full, ph) || !ptx::mbar_wait(in_full, ph) ||
            !ptx::mbar_wait_cluster(fwd_own, ph)) {
          atomicCAS(fa.err, 0, 2);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int kc = 4; kc < nk; ++kc) chunk_mmas(kc, first);
        // K-chunks 0-3: leader half local, peer half copied in from the leader
        if (!ptx::mbar_wait_cluster(fwd_in, ph)) {
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
      for (int l = 1; l <= L; ++l) {
        const uint32_t ph = (l - 1) & 1;
        if (!ptx::mbar_wait(own_full, ph)) {
          atomicCAS(fa.err, 0, 5);
          break;
        }
        ptx::mbar_arrive_cluster(own_leader);
        if (!ptx::mbar_wait(in_full, ph)) {
          atomicCAS(fa.err, 0, 6);
          break;
        }
        ptx::mbar_arrive_cluster(in_leader);
      }
    }
  } else {
    // ---- epilogue, both CTAs
    const bool own = static_cast<uint32_t>(h) == rank;   // warp-uniform
    // Destination of this thread's positions (dim d, chain rows 0-31 of half
    // h): this CTA's tile if the chains are ours, else staging, laid out as
    // K-chunks 4 rank .. 4 rank + 3 of the peer's tile (1024-byte aligned both
    // sides, so the swizzle carries over).  Row i's byte offset is
    // col + (i / 8) * 1024 + sw[i % 8]; the eight sw terms are per thread.
    const int dcol = own ? d : d - static_cast<int>(rank) * 128;
    const uint32_t col = static_cast<uint32_t>((dcol >> 5) * kBChunk + (dcol & 3) * 4);
    const uint32_t dst_hi0 = ptx::smem_u32(own ? Bhi : Stg) + col;
    const uint32_t lo_off = own ? kBBytes : kStageHalf;
    const uint32_t buf_off = own ? 0u : kStageBytes;       // staging double buffer stride
    uint32_t sw[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) sw[r] = r * 128 + (((((dcol & 31) >> 2) ^ r) & 7) << 4);
    const int nvalid = dvalid ? min(kHalf, C - (pair_base + h * kHalf)) : 0;
    auto store_x = [&](int i, float xi, int buf) {   // position of row i, split
      if (i < nvalid) {
        float hi, lo;
        split_tf32(xi, hi, lo);
        const uint32_t a0 = dst_hi0 + buf * buf_off + (i >> 3) * 1024 + sw[i & 7];
        asm volatile("st.shared.f32 [%0], %1;" ::"r"(a0), "f"(hi) : "memory");
        asm volatile("st.shared.f32 [%0], %1;" ::"r"(a0 + lo_off), "f"(lo) : "memory");
      }
    };
    // The next positions are written: own warps arrive on this CTA's tile
    // barrier (one arms the peer's incoming copy bytes); each staging warp
    // pushes its K-chunk -- staging chunk `quarter`, the peer's K-chunk
    // 4 rank + quarter -- completing on the peer's barrier.
    auto publish = [&](int buf) {
      proxy_fence_cta();          // generic stores -> async proxy (MMA, bulk copy)
      ptx::tc_fence_before();     // this thread's accumulator reads precede the next MMA
      ptx::mbar_arrive_local(own_full);
      if (own) {
        if ((ew & 3) == 0 && lane == 0) ptx::mbar_arrive_expect_tx(in_full, kStageBytes);
      } else {
        __syncwarp();
        if (lane == 0) {
          const uint32_t bar = ptx::mapa(ptx::smem_u32(in_full), peer);
          const uint32_t chunk = (4 * rank + quarter) * kBChunk;
          uint8_t* sb = Stg + buf * kStageBytes + quarter * kBChunk;
          ptx::bulk_copy_to_cluster(ptx::mapa(ptx::smem_u32(Bhi + chunk), peer), sb, kBChunk, bar);
          ptx::bulk_copy_to_cluster(ptx::mapa(ptx::smem_u32(Blo + chunk), peer), sb + kStageHalf, kBChunk, bar);
        }
      }
    };
    const uint32_t acc_addr = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + kColAcc + h * kHalf;
    auto wait_acc = [&](int l) {
      if (!ptx::mbar_wait(acc_full, (l - 1) & 1)) {
        atomicCAS(fa.err, 0, 4);
        ok = false;
      }
      ptx::tc_fence_after();
    };
    // P rows of this CTA (row = output dim d = TMEM lane) into tensor memory
    // from the pre-arranged image (coalesced): the two warps of a lane
    // quarter split chunks 0-3 and 4-6
    {
      const int kc_end = min(nk, kTmemChunks);
      for (int kc = h == 0 ? 0 : 4; kc < (h == 0 ? min(kc_end, 4) : kc_end); ++kc) {
#pragma unroll
        for (int q16 = 0; q16 < 2; ++q16) {
          float vh[16], vl[16];
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const float4 u = *reinterpret_cast<const float4*>(
                fa.Ptm + image_index(static_cast<int>(rank), kc, 0, q16, quarter, q4, lane));
            const float4 w = *reinterpret_cast<const float4*>(
                fa.Ptm + image_index(static_cast<int>(rank), kc, 1, q16, quarter, q4, lane));
            vh[4 * q4] = u.x; vh[4 * q4 + 1] = u.y; vh[4 * q4 + 2] = u.z; vh[4 * q4 + 3] = u.w;
            vl[4 * q4] = w.x; vl[4 * q4 + 1] = w.y; vl[4 * q4 + 2] = w.z; vl[4 * q4 + 3] = w.w;
          }
          const uint32_t tcol = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + kColP + 64 * kc + 16 * q16;
          ptx::tmem_st16(tcol, vh);
          ptx::tmem_st16(tcol + 32, vl);
        }
      }
      ptx::tmem_wait_st();
    }
    // begin: p = p0 + eps/2 g0, x1 = x0 + eps p
#pragma unroll
    for (int i8 = 0; i8 < kHalf; i8 += 8) {
      float xr[8], gr[8], zr[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int chain = pair_base + h * kHalf + i8 + k;
        const bool valid = i8 + k < nvalid;
        const int64_t e = static_cast<int64_t>(chain) * D + d;
        xr[k] = valid ? a.x[e] : 0.f;
        gr[k] = valid ? a.g[e] : 0.f;
        zr[k] = valid ? fa.p0[e] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = i8 + k;
        p[i] = fmaf(0.5f * eps, gr[k], zr[k]);
        x[i] = fmaf(eps, p[i], xr[k]);
        store_x(i, x[i], 0);
      }
    }
    publish(0);
    // steps 1 .. L-1: merged kick + drift
    for (int l = 1; l < L; ++l) {
      wait_acc(l);
#pragma unroll
      for (int cb = 0; cb < kHalf / 16; ++cb) {
        float accv[16];
        ptx::tmem_ld16(acc_addr + cb * 16, accv);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int i = cb * 16 + k;
          p[i] = fmaf(-eps, accv[k], p[i]);
          x[i] = fmaf(eps, p[i], x[i]);
          store_x(i, x[i], l & 1);
        }
      }
      publish(l & 1);
    }
    // step L: final half kick
    wait_acc(L);
#pragma unroll
    for (int cb = 0; cb < kHalf / 16; ++cb) {
      float accv[16];
      ptx::tmem_ld16(acc_addr + cb * 16, accv);
#pragma unroll
      for (int k = 0; k < 16; ++k) p[cb * 16 + k] = fmaf(-0.5f * eps, accv[k], p[cb * 16 + k]);
    }
    // partial sums over this CTA's dims: <x, g> and |p|^2 per chain
#pragma unroll
    for (int cb = 0; cb < kHalf / 16; ++cb) {
      float accv[16];
      ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + h * kHalf + cb * 16, accv);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int i = cb * 16 + k;
        const bool valid = dvalid && pair_base + h * kHalf + i < C;
        float xg = valid ? -x[i] * accv[k] : 0.f;
        float pp = valid ? p[i] * p[i] : 0.f;
        xg = warp_sum(xg);
        pp = warp_sum(pp);
        if (lane == 0) {
          red[(0 * 4 + quarter) * 64 + h * kHalf + i] = xg;
          red[(1 * 4 + quarter) * 64 + h * kHalf + i] = pp;
        }
      }
    }
    epi_barrier();
    const int c = ew * 32 + lane;                 // 0..255; chains 0..63 handled below
    if (c < kPairChains) {
      float xg = 0.f, pp = 0.f;
      for (int q = 0; q < 4; ++q) {
        xg += red[(0 * 4 + q) * 64 + c];
        pp += red[(1 * 4 + q) * 64 + c];
      }
      if (rank == 0) {
        red_pair[c] = xg;
        red_pair[64 + c] = pp;
      } else {
        ptx::st_cluster_f32(ptx::mapa(ptx::smem_u32(&peer_in[c]), 0), xg);
        ptx::st_cluster_f32(ptx::mapa(ptx::smem_u32(&peer_in[64 + c]), 0), pp);
      }
    }
  }
  // every copy into this CTA's tile has landed (immediate unless a wait gave up)
  if (warp == 1 && lane == 0) ptx::mbar_wait(in_full, (L - 1) & 1);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();      // the peer's partial sums have landed in the leader
  if (rank == 0 && threadIdx.x < kPairChains) {
    const int c = threadIdx.x;
    const int chain = pair_base + c;
    float prob = 0.f;
    int acc = 0;
    if (chain < C) {
      const float xg = red_pair[c] + peer_in[c];
      const float pp = red_pair[64 + c] + peer_in[64 + c];
      const float lp0 = a.lp[chain];
      const float lp1 = 0.5f * xg;
      float la = (-lp0 + fa.kin0[chain]) - (-lp1 + 0.5f * pp);
      if (!isfinite(la)) la = -INFINITY;
      const uint32_t gchain = static_cast<uint32_t>(chain) + a.chain_offset;
      acc = accept_log_uniform(a.seed, gchain, a.t) < la;
      prob = accept_prob(la);
      if (ok) {
        if (acc) a.lp[chain] = lp1;
        a.is_accepted[chain] = static_cast<uint8_t>(acc);
        a.log_accept[chain] = la;
        if (a.trace_acc) a.trace_acc[chain] = static_cast<uint8_t>(acc);
      }
    }
    acc_flag[c] = acc;
    ptx::st_cluster_s32(ptx::mapa(ptx::smem_u32(&acc_flag[c]), 1), acc);
    prob_s[c] = prob;
    if (blockIdx.x == 0 && c == 0 && a.trace_eps && ok) a.trace_eps[0] = eps;
  }
  ptx::cluster_sync();      // decisions visible in both CTAs
  if (warp >= 2) {
#pragma unroll
    for (int cb = 0; cb < kHalf / 16; ++cb) {
      float accv[16];
      ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + h * kHalf + cb * 16, accv);
      if (ok && dvalid) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int i = cb * 16 + k;
          const int chain = pair_base + h * kHalf + i;
          if (chain >= C) continue;
          const int64_t e = static_cast<int64_t>(chain) * D + d;
          if (acc_flag[h * kHalf + i]) {
            a.x[e] = x[i];
            a.g[e] = -accv[k];
            if (a.sample_out) a.sample_out[e] = x[i];
          } else if (a.sample_out) {
            a.sample_out[e] = a.x[e];
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, kTmemCols);
  }
  ptx::cluster_sync();
  double sum = 0.0;
  if (threadIdx.x == 0 && rank == 0)
    for (int c = 0; c < kPairChains; ++c) sum += static_cast<double>(prob_s[c]);
  block_partial_then_da(a.da, a.partials, sum, C, a.t_full);
}

}  // namespace

unsigned gauss_pair_grid(int64_t C) {
  return static_cast<unsigned>(2 * ((C + kPairChains - 1) / kPairChains));
}

cudaError_t launch_gauss_pair_image(const float* Phi, const float* Plo, int D, float* image,
                                    cudaStream_t s) {
  static_assert(kGaussPairImageFloats == 2 * kTmemChunks * 2 * 2 * 4 * 4 * 32 * 4, "image size");
  k_tmem_image<<<static_cast<unsigned>(kGaussPairImageFloats / 4 / 256), 256, 0, s>>>(Phi, Plo, D, image);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gauss_pair_setup() {
  return cudaFuncSetAttribute(k_gauss_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kSmem));
}

cudaError_t launch_gauss_pair_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                         KernelTimer* timer) {
  cudaError_t em = launch_gauss_momentum(a, tc, s);     // p0 and |p0|^2 / 2 of transition t
  if (em != cudaSuccess) return em;
  PairArgs fa{a, tc.err, tc.p, tc.h0, tc.Ptm};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gauss_pair_grid(a.C));
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
  if (timer) timer->begin(s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_gauss_pair, tc.mPhi128, tc.mPlo128, fa);
  if (timer) timer->end(s);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace hmc
