// ck_device.cuh -- device helpers: complex arithmetic, mbarrier / bulk-copy
// PTX wrappers with bounded waits, and the status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "conker.h"

namespace ck {

// complex add and subtract as one packed FP32x2 add (each lane rounded as
// the scalar add; a - b = a + (-b) exactly)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 cmul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Record the first error code in the plan's status word.
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A bounded wait gives up after this many nanoseconds of wall time.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the asynchronous (bulk-copy) proxy.
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; give up after
// limit_ns of wall time, record CK_ERR_TIMEOUT and return false.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, int* status, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) {
      set_status(status, CK_ERR_TIMEOUT);
      return false;
    }
  }
}

// The same with the default limit, kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
  return mbar_wait_for(bar, parity, status, kWaitLimitNs);
}

// Bulk (non-tensor) asynchronous copy global -> shared, completing on `bar`.
// Both addresses 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// The cells a summation visits: every cell [0, nc), or, with a support box
// {x0, x1, y0, y1, z0, z1} (W_0 = 0 outside it), the planes z0..z1, a
// contiguous range of whole planes of `plane` cells.
struct CellRange {
  int64_t lo, hi;
};

// Planes (or rows) lo .. hi of a box bound pair: 0 when lo > hi (an empty
// box is stored as lo = INT_MAX, hi = INT_MIN, whose difference overflows).
__host__ __device__ __forceinline__ int box_len(int lo, int hi) { return hi >= lo ? hi - lo + 1 : 0; }

__device__ __forceinline__ CellRange box_cells(const int* box, int64_t plane, int64_t nc) {
  if (!box) return CellRange{0, nc};
  const int z0 = box[4], z1 = box[5];
  if (z1 < z0) return CellRange{0, 0};
  const int64_t hi = (int64_t)(z1 + 1) * plane;
  return CellRange{(int64_t)z0 * plane, hi < nc ? hi : nc};
}

// Split k of `splits` equal parts of the range, each a multiple of `align`
// cells (the first cell of a part keeps the range's alignment).
__device__ __forceinline__ void split_cells(CellRange r, int splits, int64_t align, int k, int64_t* beg,
                                            int64_t* end) {
  int64_t cps = (r.hi - r.lo + splits - 1) / splits;
  cps = (cps + align - 1) / align * align;
  const int64_t b = r.lo + (int64_t)k * cps;
  *beg = b < r.hi ? b : r.hi;
  *end = b + cps < r.hi ? b + cps : r.hi;
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // 0 source bytes: the destination is zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}

// Copy the first n (0..16) bytes of src; the rest of the 16-byte destination is zero-filled.
__device__ __forceinline__ void cp_async16n(void* dst, const void* src, int n) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }


}  // namespace ck
