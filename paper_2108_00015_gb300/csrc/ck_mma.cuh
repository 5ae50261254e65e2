// ck_mma.cuh -- warp-level tensor-core helpers for the split-TF32 product
// sums: TF32 rounding and truncation, and the m16n8k8 TF32 MMA with FP32
// accumulation (fragment layouts: A row g / g + 8, column t / t + 4; B row
// t / t + 4, column g; D row g / g + 8, column 2t / 2t + 1, with
// g = lane / 4 and t = lane % 4).
#pragma once

#include <stdint.h>

namespace ck {

// Round to TF32 (nearest, ties away) and the TF32 remainder of x - hi.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

// D (16 x 8, FP32) += A (16 x 8, TF32, row-major) * B (8 x 8, TF32, column-major)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// x with its 13 low mantissa bits cleared: a TF32 number, x - hi exact in FP32
__device__ __forceinline__ uint32_t tf32_trunc(float x) { return __float_as_uint(x) & 0xffffe000u; }

}  // namespace ck
