// Warp-level tensor-core products (mma.sync) shared by the environment build's
// TF32 / BF16 contraction modes and the learned correction's network.
//
// Why mma.sync here and not tcgen05: the products are small (at most 128 x 64 x 64
// per site) and sit between two dependent steps of a latency-bound kernel whose
// shared memory is already taken by its QR / SVD working set. mma.sync builds its
// operand fragments in registers straight from that working set (rounding each
// element as it is loaded), with no staging copy, no TMEM allocation and no
// mbarrier round trip.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace tnmc {

// bfloat16 pair (lo in bits 0..15, hi in 16..31), each rounded to nearest even.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// float32 -> TF32 (10 explicit mantissa bits), round to nearest, ties away from zero.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_bf16_16816(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                               uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32_1688(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                              uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

enum : int32_t { TCMODE_NONE = 0, TCMODE_TF32 = 1, TCMODE_BF16 = 2 };

// One 16 x 8 tile of C = A B by one warp, float32 accumulators starting at zero:
// rows i0 .. i0 + 15 of A (M x K) and columns n0 .. n0 + 7 of B (K x N), both read
// through accessors that return 0 outside the matrices, every operand rounded to
// TF32 (MODE = TCMODE_TF32, k-steps of 8) or BF16 (TCMODE_BF16, k-steps of 16) as
// it is loaded. Lane (g = lane / 4, t = lane % 4) receives
//   c[0] = C[i0 + g][n0 + 2t],     c[1] = C[i0 + g][n0 + 2t + 1],
//   c[2] = C[i0 + g + 8][n0 + 2t], c[3] = C[i0 + g + 8][n0 + 2t + 1]
// (the PTX fragment layouts of m16n8k8 .tf32 and m16n8k16 .bf16).
template <int MODE, typename FA, typename FB>
__device__ __forceinline__ void tc_tile(float c[4], int K, int i0, int n0, int lane, FA A, FB B) {
  const int g = lane >> 2, t = lane & 3;
  c[0] = c[1] = c[2] = c[3] = 0.f;
  if constexpr (MODE == TCMODE_TF32) {
    for (int k = 0; k < K; k += 8) {
      const uint32_t a0 = to_tf32(A(i0 + g, k + t)), a1 = to_tf32(A(i0 + g + 8, k + t));
      const uint32_t a2 = to_tf32(A(i0 + g, k + t + 4)), a3 = to_tf32(A(i0 + g + 8, k + t + 4));
      const uint32_t b0 = to_tf32(B(k + t, n0 + g)), b1 = to_tf32(B(k + t + 4, n0 + g));
      mma_tf32_1688(c, a0, a1, a2, a3, b0, b1);
    }
  } else {
    for (int k = 0; k < K; k += 16) {
      const int kc = k + 2 * t;
      const uint32_t a0 = pack_bf16(A(i0 + g, kc), A(i0 + g, kc + 1));
      const uint32_t a1 = pack_bf16(A(i0 + g + 8, kc), A(i0 + g + 8, kc + 1));
      const uint32_t a2 = pack_bf16(A(i0 + g, kc + 8), A(i0 + g, kc + 9));
      const uint32_t a3 = pack_bf16(A(i0 + g + 8, kc + 8), A(i0 + g + 8, kc + 9));
      const uint32_t b0 = pack_bf16(B(kc, n0 + g), B(kc + 1, n0 + g));
      const uint32_t b1 = pack_bf16(B(kc + 8, n0 + g), B(kc + 9, n0 + g));
      mma_bf16_16816(c, a0, a1, a2, a3, b0, b1);
    }
  }
}

}  // namespace tnmc
