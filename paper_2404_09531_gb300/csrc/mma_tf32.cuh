// mma_tf32.cuh -- FP32-accurate matrix products on tensor cores for the
// deferred MLP (Eq. 4): mma.sync m16n8k8 TF32 with each operand split into
// a TF32 part and a TF32 residual, c += A_lo B_hi + A_hi B_lo + A_hi B_hi
// (the dropped A_lo B_lo term is below FP32 rounding), FP32 accumulation.
//
// Fragment layout (g = lane / 4, t = lane % 4): A (16 x 8) a0 = A[g][t],
// a1 = A[g + 8][t], a2 = A[g][t + 4], a3 = A[g + 8][t + 4]; B (8 x 8) b0 =
// B[t][g], b1 = B[t + 4][g]; C (16 x 8) c0 = C[g][2t], c1 = C[g][2t + 1],
// c2 = C[g + 8][2t], c3 = C[g + 8][2t + 1].
#pragma once

#include "common.cuh"

namespace omerf {

__device__ __forceinline__ void split_tf32(float v, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(v));
  const float r = v - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c += A . B with A = (ah + al), B = (b0, b1) split here: three TF32 products.
__device__ __forceinline__ void mma3(float c[4], const uint32_t ah[4], const uint32_t al[4], float b0, float b1) {
  uint32_t bh0, bl0, bh1, bl1;
  split_tf32(b0, bh0, bl0);
  split_tf32(b1, bh1, bl1);
  mma_tf32(c, al, bh0, bh1);
  mma_tf32(c, ah, bl0, bl1);
  mma_tf32(c, ah, bh0, bh1);
}

// Split the A fragment (rows r0 / r1 = m-tile rows g / g + 8, columns c0 and
// c0 + 4 of the staged rows, zero where the column is not valid).
__device__ __forceinline__ void load_a(const float* r0, const float* r1, int c0, bool v0, bool v1, uint32_t ah[4],
                                       uint32_t al[4]) {
  split_tf32(v0 ? r0[c0] : 0.0f, ah[0], al[0]);
  split_tf32(v0 ? r1[c0] : 0.0f, ah[1], al[1]);
  split_tf32(v1 ? r0[c0 + 4] : 0.0f, ah[2], al[2]);
  split_tf32(v1 ? r1[c0 + 4] : 0.0f, ah[3], al[3]);
}

}  // namespace omerf
