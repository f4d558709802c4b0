// Batched target log-prob and gradient kernels ("list of vectors" evaluation,
// Section 2.1): every chain is one row, only the event axis is reduced, so a
// chain's result never depends on another chain's.
//
//   STD_NORMAL  lp = -|x|^2/2, g = -x                      (warp per chain)
//   FUNNEL      closed form with one row reduction          (warp per chain)
//   CORR_GAUSS  G = -X P as one C x D x D product, lp = <x, g>/2
//   LOGREG      Z = Theta X^T (C x N x D), R = y - sigmoid(Z) fused into the
//               product's epilogue with the per-tile sums of y z - softplus(z);
//               G = R X - Theta (C x D x N, split over N); lp from the partials.
//
// These are the general-purpose kernels: the plain sampler calls them once per
// leapfrog step and the public gradient entry point uses them directly.
#include <cmath>

#include "hmc_device.cuh"
#include "hmc_internal.h"

namespace hmc {

std::atomic<uint64_t> g_launches{0};

// SM count of the current device (the logistic regression's split-K and
// path decisions); 152, a GB300's count, when no device can be queried.
int current_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return 152;
  }
  return sms;
}


namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

// ---------------------------------------------------------------- SIMT GEMM
// acc[i][j] for row m0 + ty + 16 i, column n0 + tx + 16 j of A[M x K] * B,
// summed over k in [k_begin, k_end).  B_NT selects B stored [N x K] row-major
// (the product uses B^T); otherwise B is [K x N] row-major.
template <bool B_NT>
__device__ __forceinline__ void gemm_tile(const float* __restrict__ A, int64_t lda,
                                          const float* __restrict__ B, int64_t ldb, int M, int N,
                                          int k_begin, int k_end, int m0, int n0,
                                          float acc[4][4]) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = k_begin; k0 < k_end; k0 += kBK) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = tid + kGemmThreads * it;
      {
        const int r = idx >> 4, kk = idx & 15;
        const int m = m0 + r, k = k0 + kk;
        As[kk][r] = (m < M && k < k_end) ? A[static_cast<int64_t>(m) * lda + k] : 0.f;
      }
      if (B_NT) {
        const int c = idx >> 4, kk = idx & 15;
        const int n = n0 + c, k = k0 + kk;
        Bs[kk][c] = (n < N && k < k_end) ? B[static_cast<int64_t>(n) * ldb + k] : 0.f;
      } else {
        const int kk = idx >> 6, c = idx & 63;
        const int n = n0 + c, k = k0 + kk;
        Bs[kk][c] = (n < N && k < k_end) ? B[static_cast<int64_t>(k) * ldb + n] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// G = -X P  (corr_gauss; P symmetric so B may be read either way)
__global__ void __launch_bounds__(kGemmThreads)
k_corr_gauss_grad(int C, int D, const float* __restrict__ x, const float* __restrict__ P,
                  float* __restrict__ g) {
  float acc[4][4];
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  gemm_tile<false>(x, D, P, D, C, D, 0, D, m0, n0, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= C) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n < D) g[static_cast<int64_t>(m) * D + n] = -acc[i][j];
    }
  }
}

// lp[c] = <x_c, g_c> / 2, warp per chain
__global__ void k_half_rowdot(int C, int D, const float* __restrict__ x,
                              const float* __restrict__ g, float* __restrict__ lp) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  const float* xr = x + static_cast<int64_t>(c) * D;
  const float* gr = g + static_cast<int64_t>(c) * D;
  float s = 0.f;
  for (int d = lane; d < D; d += 32) s = fmaf(xr[d], gr[d], s);
  s = warp_sum(s);
  if (lane == 0) lp[c] = 0.5f * s;
}

__device__ __forceinline__ float stable_sigmoid(float z) {
  const float e = expf(-fabsf(z));
  return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}

__device__ __forceinline__ float stable_softplus(float z) {
  return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
}

// Z = Theta X^T; R = y - sigmoid(Z); lp_part[c, tile] = sum_tile (y z - softplus z)
__global__ void __launch_bounds__(kGemmThreads)
k_logreg_residual(int C, int D, int N, const float* __restrict__ th, const float* __restrict__ X,
                  const float* __restrict__ y, float* __restrict__ R, float* __restrict__ lp_part) {
  float acc[4][4];
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  gemm_tile<true>(th, D, X, D, C, N, 0, D, m0, n0, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int ntiles = gridDim.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    float part = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (m < C && n < N) {
        const float z = acc[i][j], yn = y[n];
        R[static_cast<int64_t>(m) * N + n] = yn - stable_sigmoid(z);
        part += yn * z - stable_softplus(z);
      }
    }
    // the 16 threads sharing ty are one half-warp: reduce across tx
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (tx == 0 && m < C) lp_part[static_cast<int64_t>(m) * ntiles + blockIdx.x] = part;
  }
}

// Gpart[s] = R[:, chunk s] X[chunk s, :]
__global__ void __launch_bounds__(kGemmThreads)
k_logreg_grad_partial(int C, int D, int N, int chunk, const float* __restrict__ R,
                      const float* __restrict__ X, float* __restrict__ Gpart) {
  float acc[4][4];
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int kb = blockIdx.z * chunk, ke = min(N, kb + chunk);
  gemm_tile<false>(R, N, X, D, C, D, kb, ke, m0, n0, acc);
  float* out = Gpart + static_cast<int64_t>(blockIdx.z) * C * D;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= C) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n < D) out[static_cast<int64_t>(m) * D + n] = acc[i][j];
    }
  }
}

// g = sum_s Gpart[s] - theta; lp = sum_tiles lp_part - |theta|^2/2 (warp per chain)
__global__ void k_logreg_finalize(int C, int D, int splits, int ntiles, const float* __restrict__ th,
                                  const float* __restrict__ Gpart, const float* __restrict__ lp_part,
                                  float* __restrict__ g, float* __restrict__ lp) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  const int64_t row = static_cast<int64_t>(c) * D;
  float sq = 0.f;
  for (int d = lane; d < D; d += 32) {
    const float t = th[row + d];
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += Gpart[static_cast<int64_t>(s) * C * D + row + d];
    g[row + d] = acc - t;
    sq = fmaf(t, t, sq);
  }
  float part = 0.f;
  for (int k = lane; k < ntiles; k += 32) part += lp_part[static_cast<int64_t>(c) * ntiles + k];
  sq = warp_sum(sq);
  part = warp_sum(part);
  if (lane == 0) lp[c] = part - 0.5f * sq;
}

__global__ void k_std_normal_grad(int C, int D, const float* __restrict__ x, float* __restrict__ lp,
                                  float* __restrict__ g) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  const int64_t row = static_cast<int64_t>(c) * D;
  float s = 0.f;
  for (int d = lane; d < D; d += 32) {
    const float v = x[row + d];
    g[row + d] = -v;
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if (lane == 0) lp[c] = -0.5f * s;
}

__global__ void k_funnel_grad(int C, int D, const float* __restrict__ x, float* __restrict__ lp,
                              float* __restrict__ g) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  const int64_t row = static_cast<int64_t>(c) * D;
  const float v = x[row];
  float q = 0.f;
  for (int d = 1 + lane; d < D; d += 32) q = fmaf(x[row + d], x[row + d], q);
  q = warp_sum(q);
  const float ev = expf(-v);
  const float half_n = 0.5f * static_cast<float>(D - 1);
  for (int d = 1 + lane; d < D; d += 32) g[row + d] = -ev * x[row + d];
  if (lane == 0) {
    g[row] = -v / 9.f - half_n + 0.5f * ev * q;
    lp[c] = -v * v / 18.f - half_n * v - 0.5f * ev * q;
  }
}

struct LogregPlan {
  int ntiles_n;   // column tiles of the C x N residual product
  int splits;     // split of the N reduction in G = R X
  int chunk;      // rows of X per split (multiple of kBK)
  size_t off_R, off_G, off_lp, bytes;
};

inline size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

LogregPlan logreg_plan(int64_t C, int D, int64_t N) {
  LogregPlan p{};
  p.ntiles_n = static_cast<int>((N + kBN - 1) / kBN);
  const int64_t out_tiles = ((C + kBM - 1) / kBM) * ((D + kBN - 1) / kBN);
  int64_t s = (4 * static_cast<int64_t>(current_sm_count()) + out_tiles - 1) / out_tiles;
  s = std::max<int64_t>(1, std::min<int64_t>(s, (N + 511) / 512));
  int64_t chunk = (N + s - 1) / s;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  s = (N + chunk - 1) / chunk;
  p.splits = static_cast<int>(s);
  p.chunk = static_cast<int>(chunk);
  p.off_R = 0;
  p.off_G = align256(sizeof(float) * C * N);
  p.off_lp = p.off_G + align256(sizeof(float) * s * C * D);
  p.bytes = p.off_lp + align256(sizeof(float) * C * p.ntiles_n);
  return p;
}

inline unsigned warps_grid(int64_t C, int warps_per_block) {
  return static_cast<unsigned>((C + warps_per_block - 1) / warps_per_block);
}

// dx[c, :] = w[c] * g[c, :]   (vector-Jacobian product of log p)
__global__ void k_scale_rows(int C, int D, const float* __restrict__ w, float* __restrict__ g) {
  const int64_t n = static_cast<int64_t>(C) * D;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    g[i] *= w[i / D];
}

}  // namespace

cudaError_t launch_vjp(const hmc_target& t, int64_t C, const float* x, const float* w, float* dx,
                       float* lp_tmp, void* ws, cudaStream_t s) {
  cudaError_t e = launch_grad(t, C, x, lp_tmp, dx, ws, s);
  if (e != cudaSuccess) return e;
  const int64_t n = C * t.dim;
  k_scale_rows<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 152 * 16)), 256, 0, s>>>(
      static_cast<int>(C), t.dim, w, dx);
  count_launch();
  return cudaGetLastError();
}

size_t grad_workspace_bytes(const hmc_target& t, int64_t C) {
  if (t.id == HMC_T_LOGREG) return logreg_plan(C, t.dim, t.n_data).bytes;
  return 0;
}

cudaError_t launch_grad(const hmc_target& t, int64_t C64, const float* x, float* lp, float* g,
                        void* ws, cudaStream_t s, KernelTimer* timer) {
  const int C = static_cast<int>(C64), D = t.dim;
  switch (t.id) {
    case HMC_T_STD_NORMAL:
      k_std_normal_grad<<<warps_grid(C, 8), 256, 0, s>>>(C, D, x, lp, g);
      count_launch();
      break;
    case HMC_T_FUNNEL:
      k_funnel_grad<<<warps_grid(C, 8), 256, 0, s>>>(C, D, x, lp, g);
      count_launch();
      break;
    case HMC_T_CORR_GAUSS: {
      dim3 grid((D + kBN - 1) / kBN, (C + kBM - 1) / kBM);
      if (timer) timer->begin(s);
      k_corr_gauss_grad<<<grid, kGemmThreads, 0, s>>>(C, D, x, t.P, g);
      if (timer) timer->end(s);
      k_half_rowdot<<<warps_grid(C, 8), 256, 0, s>>>(C, D, x, g, lp);
      count_launch(2);
      break;
    }
    case HMC_T_LOGREG: {
      const int N = static_cast<int>(t.n_data);
      const LogregPlan p = logreg_plan(C, D, N);
      char* base = static_cast<char*>(ws);
      float* R = reinterpret_cast<float*>(base + p.off_R);
      float* Gp = reinterpret_cast<float*>(base + p.off_G);
      float* lpp = reinterpret_cast<float*>(base + p.off_lp);
      dim3 g1(p.ntiles_n, (C + kBM - 1) / kBM);
      if (timer) timer->begin(s);
      k_logreg_residual<<<g1, kGemmThreads, 0, s>>>(C, D, N, x, t.X, t.y, R, lpp);
      dim3 g2((D + kBN - 1) / kBN, (C + kBM - 1) / kBM, p.splits);
      k_logreg_grad_partial<<<g2, kGemmThreads, 0, s>>>(C, D, N, p.chunk, R, t.X, Gp);
      if (timer) timer->end(s);
      k_logreg_finalize<<<warps_grid(C, 8), 256, 0, s>>>(C, D, p.splits, p.ntiles_n, x, Gp, lpp,
                                                         g, lp);
      count_launch(3);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hmc
