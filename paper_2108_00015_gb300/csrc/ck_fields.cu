// ck_fields.cu -- fields given on the grid instead of catalogs, and per-cell
// product maps.
//  * field_load_kernel: a caller's field in box layout (x fastest) into a
//    plan field in the stored layout (the box, or the corner of its
//    zero-padded transform grid): a copy (cross-correlation maps, Sec. 2.8),
//    or the continuous over-density of Eq. 15, delta = (D - R) / R where
//    R > 0 and 0 where R <= 0 (no survey there).  One warp per row of cells;
//    the nonzero cells' count and bounding box go to the plan state (block
//    reduced, then atomics), for the guard band of a box plan.
//  * field_check_kernel: the guard band over the loaded fields (both load
//    into field 0's extent: their nonzero cells plus the kernels' reach must
//    stay inside the transformed grid on each axis).
//  * product_map_kernel: W_0 W_s / <B_0 B_s> per cell of the box (the maps
//    of Sec. 4.2), <B_0 B_s> = alpha^2 den_raw_2(s) / N_box, the average of
//    the random field's order-2 terms over the box.
#include <limits.h>
#include <stdint.h>

#include <algorithm>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {

namespace {

constexpr int FL_THREADS = 256;

struct Layout {
  int n[3];    // the box
  int dim[3];  // the stored grid
};

__global__ void __launch_bounds__(FL_THREADS) field_load_kernel(Layout L, const float* __restrict__ a,
                                                                const float* __restrict__ b, int delta,
                                                                float* __restrict__ out, DevState* st,
                                                                int which) {
  const int lane = threadIdx.x & 31;
  const unsigned nrows = (unsigned)L.n[1] * (unsigned)L.n[2];
  const unsigned wstride = gridDim.x * (blockDim.x >> 5);
  unsigned long long kept = 0;
  int bmin[3] = {INT_MAX, INT_MAX, INT_MAX}, bmax[3] = {INT_MIN, INT_MIN, INT_MIN};
  // whole rows of 16-byte groups: row starts (box and stored) and pointers aligned
  const bool vec = (L.n[0] & 3) == 0 && (L.dim[0] & 3) == 0 && ((uintptr_t)a & 15) == 0 &&
                   (!b || ((uintptr_t)b & 15) == 0) && ((uintptr_t)out & 15) == 0;
  // rows by a running (iy, iz): no integer division in the loop
  unsigned row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int iy = (int)(row % (unsigned)L.n[1]), iz = (int)(row / (unsigned)L.n[1]);
  const int sy = (int)(wstride % (unsigned)L.n[1]), sz = (int)(wstride / (unsigned)L.n[1]);
  const bool use_b = delta && b;
  auto value = [&](float v, float r) { return use_b ? (r > 0.0f ? (v - r) / r : 0.0f) : v; };
  auto take = [&](float v, int ix) {
    if (v != 0.0f) {
      ++kept;
      bmin[0] = min(bmin[0], ix); bmax[0] = max(bmax[0], ix);
      bmin[1] = min(bmin[1], iy); bmax[1] = max(bmax[1], iy);
      bmin[2] = min(bmin[2], iz); bmax[2] = max(bmax[2], iz);
    }
  };
  for (; row < nrows; row += wstride) {
    const size_t src = (size_t)row * L.n[0];
    float* __restrict__ orow = out + ((size_t)iz * L.dim[1] + iy) * L.dim[0];
    if (vec) {
      // 16-byte accesses, four per lane in flight
      const float4* a4 = reinterpret_cast<const float4*>(a + src);
      const float4* b4 = reinterpret_cast<const float4*>(b + src);
      float4* o4 = reinterpret_cast<float4*>(orow);
      const int nv = L.n[0] >> 2;
      for (int j0 = 0; j0 < nv; j0 += 128) {
        float4 qa[4], qb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * 32 + lane;
          qa[u] = j < nv ? __ldg(a4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
          qb[u] = (use_b && j < nv) ? __ldg(b4 + j) : make_float4(1.f, 1.f, 1.f, 1.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * 32 + lane;
          if (j >= nv) continue;
          const float4 v = make_float4(value(qa[u].x, qb[u].x), value(qa[u].y, qb[u].y), value(qa[u].z, qb[u].z),
                                       value(qa[u].w, qb[u].w));
          o4[j] = v;
          take(v.x, 4 * j);
          take(v.y, 4 * j + 1);
          take(v.z, 4 * j + 2);
          take(v.w, 4 * j + 3);
        }
      }
    } else {
      for (int ix = lane; ix < L.n[0]; ix += 32) {
        const float v = value(__ldg(a + src + ix), use_b ? __ldg(b + src + ix) : 1.0f);
        orow[ix] = v;
        take(v, ix);
      }
    }
    iy += sy;
    iz += sz;
    if (iy >= L.n[1]) {
      iy -= L.n[1];
      ++iz;
    }
  }
  for (int off = 16; off > 0; off >>= 1) kept += __shfl_down_sync(0xFFFFFFFFu, kept, off);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    bmin[k] = __reduce_min_sync(0xFFFFFFFFu, bmin[k]);
    bmax[k] = __reduce_max_sync(0xFFFFFFFFu, bmax[k]);
  }
  __shared__ unsigned long long sk[FL_THREADS / 32];
  __shared__ int smin[FL_THREADS / 32][3], smax[FL_THREADS / 32][3];
  const int w = threadIdx.x >> 5;
  if (lane == 0) {
    sk[w] = kept;
    for (int k = 0; k < 3; ++k) { smin[w][k] = bmin[k]; smax[w][k] = bmax[k]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long K = 0;
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int j = 0; j < FL_THREADS / 32; ++j) {
      K += sk[j];
      for (int k = 0; k < 3; ++k) { mn[k] = min(mn[k], smin[j][k]); mx[k] = max(mx[k], smax[j][k]); }
    }
    if (K) {
      atomicAdd(&st->kept[which], K);
      for (int k = 0; k < 3; ++k) {
        atomicMin(&st->bbox_min[which][k], mn[k]);
        atomicMax(&st->bbox_max[which][k], mx[k]);
      }
    }
  }
}

__global__ void field_check_kernel(DevState* st, int periodic, int nx, int ny, int nz, int mx, int my, int mz) {
  if (periodic) return;
  if (!st->kept[0]) return;
  const int n[3] = {nx, ny, nz}, m[3] = {mx, my, mz};
  for (int a = 0; a < 3; ++a)
    if (st->bbox_max[0][a] - st->bbox_min[0][a] + m[a] >= n[a]) set_status(&st->status, CK_ERR_GUARD_BAND);
}

__global__ void __launch_bounds__(FL_THREADS) product_map_kernel(Layout L, const float* __restrict__ w0,
                                                                 const float* __restrict__ ws,
                                                                 const double* __restrict__ den2, double n_box,
                                                                 DevState* st, float* __restrict__ out) {
  const double a = st->alpha;
  const double avg = a * a * den2[0] / n_box;  // <B_0 B_s>
  if (!(avg > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(&st->status, CK_ERR_ZERO_DENOM);
  }
  const float inv = avg > 0.0 ? (float)(1.0 / avg) : __int_as_float(0x7fc00000);
  const bool vec = (L.n[0] & 3) == 0 && (L.dim[0] & 3) == 0 && ((uintptr_t)w0 & 15) == 0 &&
                   ((uintptr_t)ws & 15) == 0 && ((uintptr_t)out & 15) == 0;
  const int lane = threadIdx.x & 31;
  const unsigned nrows = (unsigned)L.n[1] * (unsigned)L.n[2];
  const unsigned wstride = gridDim.x * (blockDim.x >> 5);
  unsigned row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int iy = (int)(row % (unsigned)L.n[1]), iz = (int)(row / (unsigned)L.n[1]);
  const int sy = (int)(wstride % (unsigned)L.n[1]), sz = (int)(wstride / (unsigned)L.n[1]);
  for (; row < nrows; row += wstride) {
    const size_t cell = ((size_t)iz * L.dim[1] + iy) * L.dim[0];
    float* __restrict__ orow = out + (size_t)row * L.n[0];
    if (vec) {
      const float4* a4 = reinterpret_cast<const float4*>(w0 + cell);
      const float4* b4 = reinterpret_cast<const float4*>(ws + cell);
      float4* o4 = reinterpret_cast<float4*>(orow);
      const int nv = L.n[0] >> 2;
      for (int j = lane; j < nv; j += 32) {
        const float4 x = __ldg(a4 + j), y = __ldg(b4 + j);
        o4[j] = make_float4(x.x * y.x * inv, x.y * y.y * inv, x.z * y.z * inv, x.w * y.w * inv);
      }
    } else {
      for (int ix = lane; ix < L.n[0]; ix += 32) orow[ix] = __ldg(w0 + cell + ix) * __ldg(ws + cell + ix) * inv;
    }
    iy += sy;
    iz += sz;
    if (iy >= L.n[1]) {
      iy -= L.n[1];
      ++iz;
    }
  }
}

Layout layout_of(const Plan& p) {
  Layout L;
  for (int a = 0; a < 3; ++a) {
    L.n[a] = p.box_n[a];
    L.dim[a] = p.grid.n[a];
  }
  return L;
}

unsigned row_blocks(const Plan& p) {
  const int64_t rows = (int64_t)p.box_n[1] * p.box_n[2];
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + FL_THREADS / 32 - 1) / (FL_THREADS / 32),
                                                         (int64_t)p.sm_count * 8));
}

}  // namespace

void launch_field_load(const Plan& p, const float* a, const float* b, bool delta, float* out, int which,
                       cudaStream_t st) {
  const int64_t nbox = (int64_t)p.box_n[0] * p.box_n[1] * p.box_n[2];
  ProfScope ps(p, ST_PREP, (double)nbox * (4.0 * (delta && b ? 3 : 2)), st);
  field_load_kernel<<<row_blocks(p), FL_THREADS, 0, st>>>(layout_of(p), a, b, delta ? 1 : 0, out, p.dstate, which);
}

void launch_field_check(const Plan& p, cudaStream_t st) {
  field_check_kernel<<<1, 1, 0, st>>>(p.dstate, p.grid.periodic ? 1 : 0, p.grid.n[0], p.grid.n[1], p.grid.n[2],
                                      p.maxoff[0], p.maxoff[1], p.maxoff[2]);
}

void launch_product_map(const Plan& p, const float* w0, const float* ws, int shell, float* out, cudaStream_t st) {
  const int64_t nbox = (int64_t)p.box_n[0] * p.box_n[1] * p.box_n[2];
  ProfScope ps(p, ST_OTHER, 12.0 * (double)nbox, st);
  product_map_kernel<<<row_blocks(p), FL_THREADS, 0, st>>>(layout_of(p), w0, ws,
                                                           p.den_raw + p.multiset_base[2] + shell, (double)nbox,
                                                           p.dstate, out);
}

}  // namespace ck
