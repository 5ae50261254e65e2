// ck_sums.cuh -- per-cell accumulation of the product sums of Eq. 11 in
// registers: for a cell with values v[0] = W0 (the density field N) and
// v[1 + a] = W_a, add W0 W_a (n = 2), W0 W_a W_b (n = 3, a <= b), ... to
// FP32 accumulators in the packed multiset order (n = 2 block, then n = 3 in
// lexicographic (a, b) order, ...), and flush warp sums into FP64.
#pragma once

#include "ck_device.cuh"

namespace ck {

__host__ __device__ constexpr int cmb(int n, int k) {
  // C(n, k) for the small arguments used here
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

template <int NS, int MAXN>
struct RegOut {
  static constexpr int n2 = NS;
  static constexpr int n3 = MAXN >= 3 ? cmb(NS + 1, 2) : 0;
  static constexpr int n4 = MAXN >= 4 ? cmb(NS + 2, 3) : 0;
  static constexpr int n5 = MAXN >= 5 ? cmb(NS + 3, 4) : 0;
  static constexpr int total = n2 + n3 + n4 + n5;
};

template <int NS, int MAXN>
__device__ __forceinline__ void reg_accumulate(float* acc, const float* v) {
  using O = RegOut<NS, MAXN>;
  int i3 = O::n2, i4 = O::n2 + O::n3, i5 = O::n2 + O::n3 + O::n4;
#pragma unroll
  for (int a = 0; a < NS; ++a) {
    const float p1 = v[0] * v[1 + a];
    acc[a] += p1;
    if constexpr (MAXN >= 3) {
#pragma unroll
      for (int b = a; b < NS; ++b) {
        const float p2 = p1 * v[1 + b];
        acc[i3++] += p2;
        if constexpr (MAXN >= 4) {
#pragma unroll
          for (int c = b; c < NS; ++c) {
            const float p3 = p2 * v[1 + c];
            acc[i4++] += p3;
            if constexpr (MAXN >= 5) {
#pragma unroll
              for (int d = c; d < NS; ++d) acc[i5++] += p3 * v[1 + d];
            }
          }
        }
      }
    }
  }
}

template <int NOUT>
__device__ __forceinline__ void reg_flush(float* acc, double* wacc, int lane) {
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    float t = acc[o];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
    if (lane == 0) wacc[o] += (double)t;
    acc[o] = 0.0f;
  }
}

}  // namespace ck
