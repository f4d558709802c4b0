// One launch per HMC transition for the dense Gaussian target (dim <= 256):
// each CTA owns NC chains for the whole transition -- momentum draw, all L
// leapfrog steps and the Metropolis-Hastings select (Section 2.1), with the
// chains' positions resident in shared memory and momenta in registers -- so
// the only HBM traffic of a transition is reading and writing each chain's
// state once.
//
// Gradient of step l: G^T = P X^T, computed as 3xTF32 on tcgen05 tensor
// cores, M = output dims (two 128-row tiles of P), N = the CTA's NC chains,
// K = dims; A = P (tf32 head / float32 remainder, streamed from L2 by TMA in
// 128 x 32 chunks through a ring of stages), B = the chains' positions, kept
// in shared memory as head / remainder tiles in the 128-byte-swizzled K-major
// layout the MMA reads.  Accumulators live in tensor memory; the epilogue
// warps read them (one output dim per thread, NC chains per thread), apply
// the leapfrog update and write the next positions back into the B tiles.
//
// Warp roles (320 threads): warp 0 allocates tensor memory and one lane issues
// the TMA loads of P; one lane of warp 1 issues the MMAs; warps 2-9 are the
// epilogue: warp w serves tensor-memory lane quarter w % 4 of M-tile
// (w - 2) / 4, i.e. output dim d = 128 * ((w - 2) / 4) + 32 * (w % 4) + lane.
#include <cuda.h>

#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"
#include "sm100_ptx.cuh"

namespace hmc {

namespace {

constexpr int kMaxDim = 256;
constexpr int kChunks = kMaxDim / 32;
constexpr int kThreads = 320;
constexpr int kEpiThreads = 256;
constexpr uint32_t kSlot = 128 * 128;            // one 128 x 32 float tile of P: 16 KB
constexpr uint32_t kTmemCols = 512;               // accumulators + resident P head
constexpr int kAccCols = 64;                      // two M-tiles x 32 chains

// Tensor-memory column of the resident P head for (K-chunk kc, M-tile mt),
// or -1 when that chunk does not fit and is streamed like the remainder.
// Columns [0, 64) hold the accumulators; the head of M-tile 0 takes
// [64, 320) and M-tile 1's first six K-chunks take [320, 512).
__host__ __device__ constexpr int head_col(int kc, int mt) {
  return (kAccCols + mt * 256 + kc * 32 + 32 <= static_cast<int>(kTmemCols))
             ? kAccCols + mt * 256 + kc * 32
             : -1;
}

template <int NC>
struct Cfg {
  // P chunks are shared by every CTA: a cluster of kCluster CTAs loads each
  // slot once, every CTA fetching 128 / kCluster rows and multicasting them
  static constexpr int kCluster = 4;
  static constexpr uint32_t kBChunk = NC * 128;               // NC rows x 128 B
  static constexpr uint32_t kBBytes = kChunks * kBChunk;      // one of head / remainder
  static constexpr int kSlots = 8;                            // 16 KB slots in flight
  static constexpr uint32_t kSmall = 8 * (2 * kSlots + 2) + 16 + 3 * 8 * NC * 4 + 2 * NC * 4;
  static constexpr size_t kSmem = 2 * kBBytes + kSlots * kSlot + kSmall + 1024;
};

struct FusedArgs {
  StepArgs s;
  int* err;
  const float* Phi;     // P head, row-major [D x D] (resident rows come from here)
};

// Byte offset of element (row r, column k) of a K-major tile stored as
// 32-column chunks of `chunk_bytes` with the 128-byte swizzle: 16-byte unit
// index XOR (row mod 8) inside each 8-row, 1024-byte group.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k, uint32_t chunk_bytes) {
  const int kc = k >> 5, cc = k & 31;
  return kc * chunk_bytes + (r >> 3) * 1024 + (r & 7) * 128 + ((((cc >> 2) ^ (r & 7)) & 7) << 4) +
         (cc & 3) * 4;
}

__device__ __forceinline__ void proxy_fence_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

template <int NC, int CL>
__global__ void __launch_bounds__(kThreads, 1)
k_gauss_fused(const __grid_constant__ CUtensorMap mPhi, const __grid_constant__ CUtensorMap mPlo,
              FusedArgs fa) {
  using K = Cfg<NC>;
  const StepArgs& a = fa.s;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* Bhi = smem;
  uint8_t* Blo = smem + K::kBBytes;
  uint8_t* Ast = smem + 2 * K::kBBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(Ast + K::kSlots * kSlot);
  uint64_t* empty = full + K::kSlots;
  uint64_t* acc_full = empty + K::kSlots;
  uint64_t* x_ready = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(x_ready + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);        // [3][8][NC]
  int* acc_flag = reinterpret_cast<int*>(red + 3 * 8 * NC);    // [NC]
  float* prob_s = reinterpret_cast<float*>(acc_flag + NC);     // [NC]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = a.C, D = a.D, L = a.L;
  const int nk = (D + 31) >> 5;
  const int ntm = (D + 127) >> 7;
  const int c0 = blockIdx.x * NC;

  const uint32_t crank = CL > 1 ? ptx::cluster_rank() : 0u;
  constexpr uint16_t kMask = static_cast<uint16_t>((1u << CL) - 1u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < K::kSlots; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], CL);       // released by the MMA of every CTA
    }
    ptx::mbar_init(acc_full, 1);
    ptx::mbar_init(x_ready, kEpiThreads);
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&mPhi);
    ptx::prefetch_tensormap(&mPlo);
  }
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kTmemCols);
    ptx::tmem_relinquish();
  }
  // zero the position tiles: padding rows (chains >= C) and columns (dims >= D)
  for (uint32_t i = threadIdx.x; i < 2 * K::kBBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  proxy_fence_smem();
  ptx::tc_fence_before();
  __syncthreads();
  if (CL > 1) ptx::cluster_sync();        // every CTA's barriers exist before any multicast
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const float eps = a.da->eps;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer.  Per leapfrog step, for every (M-tile, K-chunk):
      // the remainder tile of P, then the head tile when it is not resident.
      int it = 0;
      for (int l = 1; l <= L && ok; ++l)
        for (int mt = 0; mt < ntm && ok; ++mt)
          for (int kc = 0; kc < nk && ok; ++kc)
            for (int part = 0; part < (head_col(kc, mt) < 0 ? 2 : 1); ++part, ++it) {
              const int s = it % K::kSlots, round = it / K::kSlots;
              if (it >= K::kSlots && !ptx::mbar_wait(&empty[s], (round - 1) & 1)) {
                atomicExch(fa.err, 1);
                ok = false;
                break;
              }
              uint8_t* st = Ast + s * kSlot;
              const void* map = part == 0 ? static_cast<const void*>(&mPlo)
                                          : static_cast<const void*>(&mPhi);
              ptx::mbar_arrive_expect_tx(&full[s], kSlot);
              if (CL == 1) {
                ptx::tma_load_2d(st, map, &full[s], kc * 32, mt * 128);
              } else {
                constexpr int kRows = 128 / CL;
                ptx::tma_load_2d_multicast(st + crank * (kSlot / CL), map, &full[s], kc * 32,
                                           mt * 128 + static_cast<int>(crank) * kRows, kMask);
              }
            }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: 3xTF32 per (M-tile, K-chunk, K-step of 8):
      // P_lo x_hi (A streamed), then P_hi x_lo and P_hi x_hi (A resident in
      // tensor memory, or streamed for the chunks that do not fit)
      constexpr uint32_t idesc = ptx::idesc_tf32(128, NC);
      int it = 0;
      for (int l = 1; l <= L && ok; ++l) {
        if (!ptx::mbar_wait(x_ready, (l - 1) & 1)) {
          atomicExch(fa.err, 1);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int mt = 0; mt < ntm && ok; ++mt) {
          const uint32_t d_tmem = tmem + mt * NC;
          for (int kc = 0; kc < nk && ok; ++kc) {
            const uint32_t bhi = ptx::smem_u32(Bhi + kc * K::kBChunk);
            const uint32_t blo = ptx::smem_u32(Blo + kc * K::kBChunk);
            const int hc = head_col(kc, mt);
            const int s_lo = it % K::kSlots;
            if (!ptx::mbar_wait(&full[s_lo], (it / K::kSlots) & 1)) {
              atomicExch(fa.err, 1);
              ok = false;
              break;
            }
            ++it;
            int s_hi = -1;
            if (hc < 0) {
              s_hi = it % K::kSlots;
              if (!ptx::mbar_wait(&full[s_hi], (it / K::kSlots) & 1)) {
                atomicExch(fa.err, 1);
                ok = false;
                break;
              }
              ++it;
            }
            ptx::tc_fence_after();
            const uint32_t alo = ptx::smem_u32(Ast + s_lo * kSlot);
            const uint32_t ahi_smem = s_hi >= 0 ? ptx::smem_u32(Ast + s_hi * kSlot) : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const uint64_t dbhi = ptx::sw128_kmajor_desc(bhi + 32 * j);
              const uint64_t dblo = ptx::sw128_kmajor_desc(blo + 32 * j);
              ptx::mma_tf32(d_tmem, ptx::sw128_kmajor_desc(alo + 32 * j), dbhi, idesc,
                            (kc | j) != 0 ? 1u : 0u);
              if (hc >= 0) {
                const uint32_t a_tmem = tmem + static_cast<uint32_t>(hc + 8 * j);
                ptx::mma_tf32_tmem_a(d_tmem, a_tmem, dblo, idesc, 1u);
                ptx::mma_tf32_tmem_a(d_tmem, a_tmem, dbhi, idesc, 1u);
              } else {
                const uint64_t dahi = ptx::sw128_kmajor_desc(ahi_smem + 32 * j);
                ptx::mma_tf32(d_tmem, dahi, dblo, idesc, 1u);
                ptx::mma_tf32(d_tmem, dahi, dbhi, idesc, 1u);
              }
            }
            if (CL == 1) ptx::mma_commit(&empty[s_lo]);
            else ptx::mma_commit_multicast(&empty[s_lo], kMask);
            if (s_hi >= 0) {
              if (CL == 1) ptx::mma_commit(&empty[s_hi]);
              else ptx::mma_commit_multicast(&empty[s_hi], kMask);
            }
          }
        }
        ptx::mma_commit(acc_full);
      }
    }
  } else {
    // ---- epilogue: one output dim d per thread, NC chains per thread
    const int ew = warp - 2;
    const int mt = ew >> 2, quarter = warp & 3;
    const int d = mt * 128 + quarter * 32 + lane;
    const bool dvalid = d < D;
    float p[NC];
    // P head rows into tensor memory: warp (M-tile mt, lane quarter) writes
    // row d of P_hi into its lane at the resident columns (zeros past dim D)
    {
      const int kmax = mt == 0 ? 256 : static_cast<int>(kTmemCols) - kAccCols - 256;
      const int kload = min(kmax, nk * 32);
      const float* __restrict__ prow = fa.Phi + static_cast<int64_t>(min(d, D - 1)) * D;
#pragma unroll 1
      for (int k0 = 0; k0 < kload; k0 += 64) {
        float v[64];
#pragma unroll
        for (int q4 = 0; q4 < 16; ++q4) {
          const int k = k0 + 4 * q4;
          const float4 w = (dvalid && k < D) ? *reinterpret_cast<const float4*>(prow + k)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
          v[4 * q4] = w.x;
          v[4 * q4 + 1] = w.y;
          v[4 * q4 + 2] = w.z;
          v[4 * q4 + 3] = w.w;
        }
#pragma unroll
        for (int q16 = 0; q16 < 4; ++q16)
          if (k0 + 16 * q16 < kload)
            ptx::tmem_st16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                               static_cast<uint32_t>(kAccCols + mt * 256 + k0 + 16 * q16),
                           v + 16 * q16);
      }
      ptx::tmem_wait_st();
    }
    // begin: p0 ~ N(0, I), K0 partials, p = p0 + eps/2 g0, x1 = x0 + eps p.
    // The loads of x0 and g0 for a group of 8 chains are issued before any
    // of them is used.
#pragma unroll
    for (int c16 = 0; c16 < NC; c16 += 8) {
      float xr[8], gr[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int chain = c0 + c16 + i;
        const bool valid = dvalid && chain < C;
        const int64_t e = static_cast<int64_t>(chain) * D + d;
        xr[i] = valid ? a.x[e] : 0.f;
        gr[i] = valid ? a.g[e] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = c16 + i;
        const int chain = c0 + c;
        const bool valid = dvalid && chain < C;
        const float z = valid ? momentum1(a.seed, static_cast<uint32_t>(d),
                                          static_cast<uint32_t>(chain) + a.chain_offset, a.t)
                              : 0.f;
        const float k2 = warp_sum(z * z);
        if (lane == 0) red[(0 * 8 + ew) * NC + c] = k2;
        p[c] = fmaf(0.5f * eps, gr[i], z);
        if (valid) {
          float hi, lo;
          split_tf32(fmaf(eps, p[c], xr[i]), hi, lo);
          const uint32_t off = sw128_offset(c, d, K::kBChunk);
          *reinterpret_cast<float*>(Bhi + off) = hi;
          *reinterpret_cast<float*>(Blo + off) = lo;
        }
      }
    }
    proxy_fence_smem();
    ptx::tc_fence_before();
    mbar_arrive(x_ready);
    for (int l = 1; l <= L; ++l) {
      const bool last = l == L;
      if (!ptx::mbar_wait(acc_full, (l - 1) & 1)) {
        atomicExch(fa.err, 1);
        ok = false;
      }
      ptx::tc_fence_after();
#pragma unroll
      for (int cb = 0; cb < NC / 16; ++cb) {
        float accv[16];
        ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + mt * NC + cb * 16, accv);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = cb * 16 + i;
          const float g = -accv[i];
          const uint32_t off = sw128_offset(c, d, K::kBChunk);
          if (!last) {
            p[c] = fmaf(eps, g, p[c]);
            if (dvalid) {
              const float x = *reinterpret_cast<const float*>(Bhi + off) +
                              *reinterpret_cast<const float*>(Blo + off);
              float hi, lo;
              split_tf32(fmaf(eps, p[c], x), hi, lo);
              *reinterpret_cast<float*>(Bhi + off) = hi;
              *reinterpret_cast<float*>(Blo + off) = lo;
            }
          } else {
            p[c] = fmaf(0.5f * eps, g, p[c]);   // g_L stays in tensor memory
          }
        }
      }
      if (!last) {
        proxy_fence_smem();
        ptx::tc_fence_before();
        mbar_arrive(x_ready);
      }
    }
    // H_L partials: <x_L, g_L> / 2 and |p_L|^2 per chain (g_L re-read from
    // the accumulator, which the last step left in tensor memory)
#pragma unroll
    for (int cb = 0; cb < NC / 16; ++cb) {
      float accv[16];
      ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + mt * NC + cb * 16, accv);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = cb * 16 + i;
        float xg = 0.f, pp = 0.f;
        if (dvalid && c0 + c < C) {
          const uint32_t off = sw128_offset(c, d, K::kBChunk);
          const float x = *reinterpret_cast<const float*>(Bhi + off) +
                          *reinterpret_cast<const float*>(Blo + off);
          xg = -x * accv[i];
          pp = p[c] * p[c];
        }
        xg = warp_sum(xg);
        pp = warp_sum(pp);
        if (lane == 0) {
          red[(1 * 8 + ew) * NC + c] = xg;
          red[(2 * 8 + ew) * NC + c] = pp;
        }
      }
    }
    epi_barrier();
    // Metropolis-Hastings, one thread per chain
    const int cidx = ew * 32 + lane;
    if (cidx < NC) {
      const int chain = c0 + cidx;
      float prob = 0.f;
      int acc = 0;
      if (chain < C) {
        float k0 = 0.f, xg = 0.f, k1 = 0.f;
        for (int w = 0; w < 8; ++w) {
          k0 += red[(0 * 8 + w) * NC + cidx];
          xg += red[(1 * 8 + w) * NC + cidx];
          k1 += red[(2 * 8 + w) * NC + cidx];
        }
        const float lp0 = a.lp[chain];
        const float lp1 = 0.5f * xg;
        float la = (-lp0 + 0.5f * k0) - (-lp1 + 0.5f * k1);
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
      acc_flag[cidx] = acc;
      prob_s[cidx] = prob;
      if (blockIdx.x == 0 && cidx == 0 && a.trace_eps && ok) a.trace_eps[0] = eps;
    }
    epi_barrier();
#pragma unroll
    for (int cb = 0; cb < NC / 16; ++cb) {
      float accv[16];
      ptx::tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + mt * NC + cb * 16, accv);
      if (ok && dvalid) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = cb * 16 + i;
          const int chain = c0 + c;
          if (chain >= C) continue;
          const int64_t e = static_cast<int64_t>(chain) * D + d;
          if (acc_flag[c]) {
            const uint32_t off = sw128_offset(c, d, K::kBChunk);
            const float x = *reinterpret_cast<const float*>(Bhi + off) +
                            *reinterpret_cast<const float*>(Blo + off);
            a.x[e] = x;
            a.g[e] = -accv[i];
            if (a.sample_out) a.sample_out[e] = x;
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
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
  // no CTA leaves while a peer may still multicast into it or arrive on it
  if (CL > 1) ptx::cluster_sync();
  // dual averaging: this block's acceptance probabilities in chain order
  double sum = 0.0;
  if (threadIdx.x == 0)
    for (int c = 0; c < NC; ++c) sum += static_cast<double>(prob_s[c]);
  block_partial_then_da(a.da, a.partials, sum, C, a.t_full);
}

}  // namespace

int gauss_fused_chains_per_cta() { return 32; }

bool gauss_fused_supported(const hmc_target& t) {
  return t.id == HMC_T_CORR_GAUSS && t.dim % 4 == 0 && t.dim <= kMaxDim;
}

// CTAs the transition launches for C chains (a whole number of clusters).
unsigned gauss_fused_grid(int64_t C) {
  constexpr int CL = Cfg<32>::kCluster;
  const int64_t ctas = (C + 31) / 32;
  return static_cast<unsigned>((ctas + CL - 1) / CL * CL);
}

cudaError_t gauss_fused_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_gauss_fused<32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg<32>::kSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gauss_fused<32, Cfg<32>::kCluster>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(Cfg<32>::kSmem));
}

cudaError_t launch_gauss_fused_transition(const StepArgs& a, GaussTc& tc, cudaStream_t s,
                                          KernelTimer* timer) {
  FusedArgs fa{a, tc.err, tc.Phi};
  constexpr int CL = Cfg<32>::kCluster;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gauss_fused_grid(a.C));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = Cfg<32>::kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (timer) timer->begin(s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_gauss_fused<32, CL>, tc.mPhi32, tc.mPlo32, fa);
  if (timer) timer->end(s);
  count_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace hmc
