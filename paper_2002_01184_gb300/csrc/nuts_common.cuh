// What both NUTS kernels (Section 2.3, the recursion unrolled) share: the
// random streams of the tree's choices, the exact-integer choice rule, the
// divergence threshold and the per-chain scratch layout.
//
// Random choices: directions from word 0 of counter (0, chain, t, 3), the
// subtree's choice at leaf k of doubling j from word k mod 4 of counter
// (k / 4, chain, t, 4 + j), the top-level choice at doubling j from counter
// (j, chain, t, 14); a choice of probability a / b is taken iff
// (2 w + 1) b < a 2^33 (exact integers).
#pragma once

#include "hmc_device.cuh"
#include "hmc_internal.h"

namespace hmc {

constexpr uint32_t kNutsTagDirection = 3u, kNutsTagSubtree = 4u, kNutsTagTop = 14u;
constexpr float kNutsDeltaMax = 1000.f;
constexpr int kNutsMaxDepth = 10;
// per-chain scratch slots of D (or the padded row length) floats:
// 0-2 left end x, p, g; 3-5 right end; 6-7 candidate x, g; 8-9 subtree
// candidate x, g; 10 + 2 (i - 1), + 1: first leaf x, p of the open span of
// 2^i leaves (i = 1 .. max_depth - 1)
constexpr int kSlotLeft = 0, kSlotRight = 3, kSlotCand = 6, kSlotSub = 8, kSlotSpan = 10;
static_assert(kSlotSpan + 2 * (kNutsMaxDepth - 1) <= kNutsSlots, "scratch slots");

__device__ __forceinline__ uint32_t nuts_word0(uint64_t seed, uint32_t w, uint32_t chain, uint32_t t,
                                               uint32_t tag) {
  return philox(make_uint4(w, chain, t, tag), static_cast<uint32_t>(seed),
                static_cast<uint32_t>(seed >> 32)).x;
}

// the subtree-choice word of leaf k of doubling j
__device__ __forceinline__ uint32_t nuts_subtree_word(uint64_t seed, uint32_t k, uint32_t chain, uint32_t t,
                                                      int j) {
  const uint4 w = philox(make_uint4(k >> 2, chain, t, kNutsTagSubtree + static_cast<uint32_t>(j)),
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  const uint32_t q = k & 3u;
  return q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
}

// probability a / b, b > 0: (2 w + 1) b < a 2^33
__device__ __forceinline__ bool nuts_take(uint32_t w, uint32_t a, uint32_t b) {
  return (2ull * w + 1ull) * b < (static_cast<unsigned long long>(a) << 33);
}

// two warp sums in one butterfly (each the same tree as warp_sum)
__device__ __forceinline__ void warp_sum2(float& u, float& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    v += __shfl_xor_sync(0xffffffffu, v, o);
  }
}

// four warp sums in one butterfly
__device__ __forceinline__ void warp_sum4(float& u, float& v, float& w, float& z) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    v += __shfl_xor_sync(0xffffffffu, v, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
}

}  // namespace hmc
