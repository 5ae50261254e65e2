// ck_grid.cu -- mapping (Sec. 2.2): nearest-grid-point histograms of the
// data and random catalogs with one 32-bit atomic per point (the L2 absorbs
// clustered catalogs' repeated cells faster than grouping them per warp
// would cost), and the field
// preparation N = D - alpha R (Eq. 8), Rt = alpha R.
//
// Cell rule: on each axis a point x (float32) is in cell k iff
// e_k <= x < e_{k+1}, e_k = fl64(origin + fl64(k * cell)).  The kernel takes
// an FP32 estimate of k and settles it against per-axis FP32 thresholds
// t_k = the smallest float32 >= e_k (built on the host in FP64), so that
// x >= e_k  <=>  x >= t_k exactly and the counts are bit-identical to an
// exact evaluation.  Points outside [t_0, t_n) on a periodic axis take an
// FP64 path and wrap k mod n; on a non-periodic grid they are dropped and
// counted.  Non-finite coordinates are dropped on both kinds of grid.
#include <float.h>
#include <math.h>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {

struct GridArgs {
  int n[3];    // the box: cells 0 .. n - 1 per axis (points outside are dropped or wrapped)
  int dim[3];  // the stored grid (the box, or its zero-padded transform grid)
  float of[3];
  float inv_g;
  double o[3];
  double g;
  int periodic;
  const float* thr[3];
};

__device__ __forceinline__ int exact_cell_fp64(float x, double o, double g) {
  const double xd = (double)x;
  long long k = (long long)floor((xd - o) / g);
  for (int it = 0; it < 8; ++it) {
    const double lo = __dadd_rn(o, __dmul_rn((double)k, g));
    const double hi = __dadd_rn(o, __dmul_rn((double)(k + 1), g));
    if (xd < lo) { --k; continue; }
    if (xd >= hi) { ++k; continue; }
    break;
  }
  return (int)k;  // callers only use it modulo n on a periodic axis
}

// Returns false if the point falls outside a non-periodic grid (or is not
// finite).
__device__ __forceinline__ bool axis_cell(float x, int a, const GridArgs& A, int* kout) {
  if (!isfinite(x)) return false;
  const int n = A.n[a];
  const float* t = A.thr[a];
  const float e = (x - A.of[a]) * A.inv_g;
  int k;
  if (e < -1.0f) k = -2;
  else if (e > (float)n + 1.0f) k = n + 1;
  else k = (int)floorf(e);
  if (k == -1 && x >= __ldg(t)) k = 0;
  if (k == n && x < __ldg(t + n)) k = n - 1;
  bool settled = false;
#pragma unroll 1
  for (int it = 0; it < 4 && k >= 0 && k < n; ++it) {
    if (x < __ldg(t + k)) { --k; continue; }
    if (x >= __ldg(t + k + 1)) { ++k; continue; }
    settled = true;
    break;
  }
  if (settled) { *kout = k; return true; }
  if (!A.periodic) return false;
  int kk = exact_cell_fp64(x, A.o[a], A.g) % n;
  if (kk < 0) kk += n;
  *kout = kk;
  return true;
}

// Counts (W = false: a 32-bit atomic on counts per point) or weights
// (W = true: each weight rounded to a multiple of 2^-32, a 64-bit atomic on
// acc per point, so the integer sums do not depend on the order of the
// atomics; a point with a non-finite weight is dropped).
template <bool W>
__device__ __forceinline__ void grid_points_body(const float* __restrict__ xs, const float* __restrict__ ys,
                                                 const float* __restrict__ zs, const float* __restrict__ ws,
                                                 int64_t npts, const GridArgs& A, uint32_t* __restrict__ counts,
                                                 long long* __restrict__ acc, DevState* st, int which) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long kept = 0, dropped = 0;
  long long qsum = 0;
  int bmin[3] = {INT_MAX, INT_MAX, INT_MAX}, bmax[3] = {INT_MIN, INT_MIN, INT_MIN};
  // the cell of one point (0xFFFFFFFF: not a real point, or outside the
  // box), with its fixed-point weight and the kept / dropped / bounds
  // bookkeeping (in: a real point)
  auto cell_of = [&](float x, float y, float z, float wt, bool in, long long* qout) -> uint32_t {
    int kx = 0, ky = 0, kz = 0;
    long long q = 0;
    if (in) {
      bool ok = axis_cell(x, 0, A, &kx) && axis_cell(y, 1, A, &ky) && axis_cell(z, 2, A, &kz);
      if constexpr (W) {
        ok = ok && isfinite(wt);
        if (ok) q = llrint((double)wt * 4294967296.0);  // exact product; nearest, ties to even
      }
      if (ok) {
        ++kept;
        qsum += q;
        bmin[0] = min(bmin[0], kx); bmax[0] = max(bmax[0], kx);
        bmin[1] = min(bmin[1], ky); bmax[1] = max(bmax[1], ky);
        bmin[2] = min(bmin[2], kz); bmax[2] = max(bmax[2], kz);
      } else {
        ++dropped;
      }
      in = ok;
    }
    *qout = q;
    return in ? (uint32_t)(((int64_t)kz * A.dim[1] + ky) * A.dim[0] + kx) : 0xFFFFFFFFu;
  };
  // one point: one atomic (integer adds give the same sums in any order)
  auto grid_one = [&](float x, float y, float z, float wt, bool in) {
    long long q = 0;
    const uint32_t cell = cell_of(x, y, z, wt, in, &q);
    if (cell == 0xFFFFFFFFu) return;
    if constexpr (W) atomicAdd(reinterpret_cast<unsigned long long*>(acc + cell), (unsigned long long)q);  // two's complement
    else atomicAdd(counts + cell, 1u);
  };
  // 16-byte aligned arrays: four consecutive points per thread and round,
  // read with one 16-byte load per coordinate.  Trip counts are
  // warp-uniform: a warp's indices share one 32-aligned block.
  int64_t done = 0;
  const uintptr_t align = reinterpret_cast<uintptr_t>(xs) | reinterpret_cast<uintptr_t>(ys) |
                          reinterpret_cast<uintptr_t>(zs) | (W ? reinterpret_cast<uintptr_t>(ws) : 0);
  if ((align & 15) == 0) {
    const int64_t nq = npts / 4, nqround = (nq + 31) / 32 * 32;
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int64_t qi = first; qi < nqround; qi += stride) {
      const bool in = qi < nq;
      const float4 X = in ? __ldg(reinterpret_cast<const float4*>(xs) + qi) : zero4;
      const float4 Y = in ? __ldg(reinterpret_cast<const float4*>(ys) + qi) : zero4;
      const float4 Z = in ? __ldg(reinterpret_cast<const float4*>(zs) + qi) : zero4;
      float4 Wt = zero4;
      if constexpr (W) Wt = in ? __ldg(reinterpret_cast<const float4*>(ws) + qi) : zero4;
      grid_one(X.x, Y.x, Z.x, Wt.x, in);
      grid_one(X.y, Y.y, Z.y, Wt.y, in);
      grid_one(X.z, Y.z, Z.z, Wt.z, in);
      grid_one(X.w, Y.w, Z.w, Wt.w, in);
    }
    done = 4 * nq;
  }
  // the rest (every point when the arrays are not 16-byte aligned): U
  // points per thread per round, whose coordinates are loaded before any is
  // gridded, so that U independent loads per thread are in flight
  constexpr int U = 4;
  const int64_t rest = npts - done, rround = (rest + 31) / 32 * 32;
  const float* xr = xs + done;
  const float* yr = ys + done;
  const float* zr = zs + done;
  const float* wr = W ? ws + done : nullptr;
  for (int64_t base = first; base < rround; base += U * stride) {
    float px[U], py[U], pz[U], pw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * stride;
      const bool in = i < rest;
      px[u] = in ? __ldg(xr + i) : 0.0f;
      py[u] = in ? __ldg(yr + i) : 0.0f;
      pz[u] = in ? __ldg(zr + i) : 0.0f;
      pw[u] = W && in ? __ldg(wr + i) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * stride;
      if (i >= rround) break;
      grid_one(px[u], py[u], pz[u], pw[u], i < rest);
    }
  }
  // block reduction of the counters and bounding boxes
  for (int off = 16; off > 0; off >>= 1) {
    kept += __shfl_down_sync(0xFFFFFFFFu, kept, off);
    dropped += __shfl_down_sync(0xFFFFFFFFu, dropped, off);
    if constexpr (W) qsum += __shfl_down_sync(0xFFFFFFFFu, qsum, off);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bmin[a] = __reduce_min_sync(0xFFFFFFFFu, bmin[a]);
    bmax[a] = __reduce_max_sync(0xFFFFFFFFu, bmax[a]);
  }
  __shared__ unsigned long long sk[8], sd[8];
  __shared__ long long sq[8];
  __shared__ int smin[8][3], smax[8][3];
  const int w = threadIdx.x >> 5;
  if (lane == 0) {
    sk[w] = kept; sd[w] = dropped; sq[w] = qsum;
    for (int a = 0; a < 3; ++a) { smin[w][a] = bmin[a]; smax[w][a] = bmax[a]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long K = 0, Dr = 0;
    long long Q = 0;
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
      K += sk[j]; Dr += sd[j]; Q += sq[j];
      for (int a = 0; a < 3; ++a) { mn[a] = min(mn[a], smin[j][a]); mx[a] = max(mx[a], smax[j][a]); }
    }
    if (K) atomicAdd(&st->kept[which], K);
    if (W && Q) atomicAdd(reinterpret_cast<unsigned long long*>(&st->wsum[which]), (unsigned long long)Q);
    if (Dr) atomicAdd(&st->dropped[which], Dr);
    if (K) {
      for (int a = 0; a < 3; ++a) {
        atomicMin(&st->bbox_min[which][a], mn[a]);
        atomicMax(&st->bbox_max[which][a], mx[a]);
      }
    }
  }
}

__global__ void __launch_bounds__(256) grid_points_kernel(const float* __restrict__ xs,
                                                          const float* __restrict__ ys,
                                                          const float* __restrict__ zs, int64_t npts,
                                                          GridArgs A, uint32_t* __restrict__ counts,
                                                          DevState* st, int which) {
  grid_points_body<false>(xs, ys, zs, nullptr, npts, A, counts, nullptr, st, which);
}

__global__ void __launch_bounds__(256) grid_points_weighted_kernel(const float* __restrict__ xs,
                                                                   const float* __restrict__ ys,
                                                                   const float* __restrict__ zs,
                                                                   const float* __restrict__ ws, int64_t npts,
                                                                   GridArgs A, long long* __restrict__ acc,
                                                                   DevState* st, int which) {
  grid_points_body<true>(xs, ys, zs, ws, npts, A, nullptr, acc, st, which);
}

// A weighted field's cells: the exact sums of the rounded weights as
// float32 (nearest), in the field's 32-bit count buffer; the field is marked
// weighted for the preparation kernels.
__global__ void weights_to_cells_kernel(const long long* __restrict__ acc, uint32_t* __restrict__ cells, int64_t nc,
                                        DevState* st, int which) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += stride)
    cells[i] = __float_as_uint((float)((double)acc[i] * 2.3283064365386962890625e-10));  // 2^-32
  if (blockIdx.x == 0 && threadIdx.x == 0) st->weighted[which] = 1;
}

// The same with the catalog read from a device descriptor, so that one
// launch (in a captured CUDA graph) serves any catalog.
__global__ void __launch_bounds__(256) grid_points_ref_kernel(const CatalogRef* __restrict__ ref, GridArgs A,
                                                              uint32_t* __restrict__ counts, DevState* st,
                                                              int which) {
  grid_points_body<false>(ref->x, ref->y, ref->z, nullptr, ref->n, A, counts, nullptr, st, which);
}

__global__ void set_catalog_ref_kernel(CatalogRef* ref, const float* x, const float* y, const float* z, int64_t n) {
  ref->x = x;
  ref->y = y;
  ref->z = z;
  ref->n = n;
}

static GridArgs grid_args(const Plan& p) {
  GridArgs A;
  for (int a = 0; a < 3; ++a) {
    A.n[a] = p.box_n[a];
    A.dim[a] = p.grid.n[a];
    A.o[a] = p.grid.origin[a];
    A.of[a] = (float)p.grid.origin[a];
    A.thr[a] = p.thr[a];
  }
  A.g = p.grid.cell;
  A.inv_g = (float)(1.0 / p.grid.cell);
  A.periodic = p.grid.periodic ? 1 : 0;
  return A;
}

void launch_set_catalog_ref(const Plan& p, const float* x, const float* y, const float* z, int64_t n,
                            cudaStream_t st) {
  set_catalog_ref_kernel<<<1, 1, 0, st>>>(p.dref, x, y, z, n);
}

void launch_grid_points_ref(const Plan& p, int which, cudaStream_t st) {
  ProfScope ps(p, ST_GRID, 0.0, st);
  grid_points_ref_kernel<<<(unsigned)(p.sm_count * 8), 256, 0, st>>>(p.dref, grid_args(p), p.counts[which],
                                                                     p.dstate, which);
}

void launch_grid_points(const Plan& p, const float* x, const float* y, const float* z, int64_t n,
                        int which, cudaStream_t st) {
  if (n <= 0) return;
  const GridArgs A = grid_args(p);
  const int64_t warps = (n + 31) / 32;
  int64_t blocks = std::min<int64_t>((warps + 7) / 8, (int64_t)p.sm_count * 8);
  if (blocks < 1) blocks = 1;
  ProfScope ps(p, ST_GRID, 12.0 * (double)n, st);
  grid_points_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, y, z, n, A, p.counts[which], p.dstate, which);
}

// alpha = kept_D / kept_R (FP64), N = D - alpha R in FP32 (one FMA), plus the
// plan-level checks (empty catalogs, guard band on a non-periodic grid).
// The cells [c0, c1) of the planes range[0] .. range[1] (plane cells each;
// empty when range[0] > range[1]): a 16-byte aligned body of 4-cell groups
// [4 q0, 4 q1) and the cells before and after it.
struct CellSpan {
  int64_t c0, c1, q0, q1;
};
__device__ __forceinline__ CellSpan plane_span(const int* range, int64_t plane) {
  CellSpan s;
  s.c0 = (int64_t)range[0] * plane;
  s.c1 = range[0] <= range[1] ? ((int64_t)range[1] + 1) * plane : s.c0;
  const int64_t a0 = min(s.c1, (s.c0 + 3) / 4 * 4);
  s.q0 = a0 / 4;
  s.q1 = max(s.q0, s.c1 / 4);
  return s;
}

__global__ void __launch_bounds__(256) clear_counts_kernel(const DevState* __restrict__ st, int which,
                                                           uint32_t* __restrict__ counts, int64_t plane, int nz) {
  int range[2] = {0, nz - 1};
  if (st->counts_known[which]) {
    range[0] = max(st->bbox_min[which][2], 0);
    range[1] = min(st->bbox_max[which][2], nz - 1);
  }
  const CellSpan sp = plane_span(range, plane);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint4* C4 = reinterpret_cast<uint4*>(counts);
  for (int64_t i = sp.q0 + t0; i < sp.q1; i += stride) C4[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t i = sp.c0 + t0; i < 4 * sp.q0; i += stride) counts[i] = 0u;
  for (int64_t i = 4 * sp.q1 + t0; i < sp.c1; i += stride) counts[i] = 0u;
}

__global__ void __launch_bounds__(256) prepare_data_kernel(const uint32_t* __restrict__ D,
                                                           const uint32_t* __restrict__ R,
                                                           float* __restrict__ field, const int* __restrict__ range,
                                                           int64_t plane, DevState* st, int periodic, int nx, int ny,
                                                           int nz, int mx, int my, int mz, double alpha_fixed) {
  const unsigned long long kd = st->kept[0], kr = st->kept[1];
  const bool wd = st->weighted[0] != 0, wr = st->weighted[1] != 0;
  // totals: counts, exact weight sums (units of 2^-32), or FP64 field totals
  auto total = [&](int k, unsigned long long kept) {
    return st->weighted[k] == 2 ? st->fsum[k]
           : st->weighted[k]    ? (double)st->wsum[k] * 2.3283064365386962890625e-10
                                : (double)kept;
  };
  const double td = total(0, kd), tr = total(1, kr);
  // a region of a decomposed catalog takes the alpha of the whole catalog
  const double alpha = alpha_fixed > 0.0 ? alpha_fixed : (tr > 0.0 ? td / tr : 0.0);
  const float af = (float)alpha;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->alpha = alpha;
    if (kd == 0 || kr == 0 || !(tr > 0.0)) set_status(&st->status, CK_ERR_EMPTY_CATALOG);
    if (!periodic && kd && kr) {
      const int n[3] = {nx, ny, nz}, m[3] = {mx, my, mz};
      for (int a = 0; a < 3; ++a) {
        const int lo = min(st->bbox_min[0][a], st->bbox_min[1][a]);
        const int hi = max(st->bbox_max[0][a], st->bbox_max[1][a]);
        if (hi - lo + m[a] >= n[a]) set_status(&st->status, CK_ERR_GUARD_BAND);
      }
    }
  }
  const CellSpan sp = plane_span(range, plane);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint4* D4 = reinterpret_cast<const uint4*>(D);
  const uint4* R4 = reinterpret_cast<const uint4*>(R);
  float4* F4 = reinterpret_cast<float4*>(field);
  // a cell: a count, or the float32 bits of a weight sum
  auto val = [](uint32_t u, bool weighted) { return weighted ? __uint_as_float(u) : (float)u; };
  for (int64_t i = sp.q0 + t0; i < sp.q1; i += stride) {
    const uint4 d = __ldg(D4 + i), r = __ldg(R4 + i);
    F4[i] = make_float4(fmaf(-af, val(r.x, wr), val(d.x, wd)), fmaf(-af, val(r.y, wr), val(d.y, wd)),
                        fmaf(-af, val(r.z, wr), val(d.z, wd)), fmaf(-af, val(r.w, wr), val(d.w, wd)));
  }
  for (int64_t i = sp.c0 + t0; i < 4 * sp.q0; i += stride) field[i] = fmaf(-af, val(R[i], wr), val(D[i], wd));
  for (int64_t i = 4 * sp.q1 + t0; i < sp.c1; i += stride) field[i] = fmaf(-af, val(R[i], wr), val(D[i], wd));
}

__global__ void __launch_bounds__(256) prepare_randoms_kernel(const uint32_t* __restrict__ R,
                                                              float* __restrict__ field,
                                                              const int* __restrict__ range, int64_t plane,
                                                              DevState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->kept[1] == 0) set_status(&st->status, CK_ERR_EMPTY_CATALOG);
  const bool wr = st->weighted[1] != 0;
  auto val = [](uint32_t u, bool weighted) { return weighted ? __uint_as_float(u) : (float)u; };
  const CellSpan sp = plane_span(range, plane);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint4* R4 = reinterpret_cast<const uint4*>(R);
  float4* F4 = reinterpret_cast<float4*>(field);
  for (int64_t i = sp.q0 + t0; i < sp.q1; i += stride) {
    const uint4 r = __ldg(R4 + i);
    F4[i] = make_float4(val(r.x, wr), val(r.y, wr), val(r.z, wr), val(r.w, wr));
  }
  for (int64_t i = sp.c0 + t0; i < 4 * sp.q0; i += stride) field[i] = val(R[i], wr);
  for (int64_t i = 4 * sp.q1 + t0; i < sp.c1; i += stride) field[i] = val(R[i], wr);
}

static unsigned elementwise_blocks(const Plan& p, int64_t n) {
  int64_t b = (n / 4 + 255) / 256;
  b = std::min<int64_t>(b, (int64_t)p.sm_count * 8);
  return (unsigned)std::max<int64_t>(b, 1);
}

// The preparations rewrite the planes support[12] .. support[13] only (the
// occupied box's, and those where the field may still be nonzero); the
// field stays exact everywhere.  Bytes: those of the box's planes.
void launch_prepare_data(const Plan& p, cudaStream_t st) {
  launch_support_box(p, 0, st);
  const int64_t plane = (int64_t)p.grid.n[0] * p.grid.n[1];
  ProfScope ps(p, ST_PREP, 0.0, 0.0, 12.0 * (double)plane, p.support + 6, st);
  prepare_data_kernel<<<elementwise_blocks(p, p.nc), 256, 0, st>>>(
      p.counts[0], p.counts[1], p.field, p.support + 12, plane, p.dstate, p.grid.periodic ? 1 : 0, p.grid.n[0],
      p.grid.n[1], p.grid.n[2], p.maxoff[0], p.maxoff[1], p.maxoff[2], p.region_alpha);
}

void launch_grid_points_weighted(const Plan& p, const float* x, const float* y, const float* z, const float* w,
                                 int64_t n, int which, cudaStream_t st) {
  if (n <= 0) return;
  const GridArgs A = grid_args(p);
  const int64_t warps = (n + 31) / 32;
  int64_t blocks = std::min<int64_t>((warps + 7) / 8, (int64_t)p.sm_count * 8);
  if (blocks < 1) blocks = 1;
  ProfScope ps(p, ST_GRID, 16.0 * (double)n, st);
  grid_points_weighted_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, y, z, w, n, A, p.wacc, p.dstate, which);
}

void launch_weights_to_cells(const Plan& p, int which, cudaStream_t st) {
  ProfScope ps(p, ST_GRID, 12.0 * (double)p.nc, st);
  weights_to_cells_kernel<<<elementwise_blocks(p, p.nc), 256, 0, st>>>(p.wacc, p.counts[which], p.nc, p.dstate,
                                                                        which);
}

// The box of cells where the field may be nonzero: the occupied cells of the
// data and the randoms (mode 0, N = D - alpha R) or of the randoms (mode 1,
// Rt); {x0, x1, y0, y1, z0, z1} inclusive, empty when a lower bound exceeds
// its upper one.  box[6..11]: that box (the forward transform's input);
// box[0..5]: the same clipped to the region's planes (where W_0 may be
// nonzero: the pruned inverse passes of the fused path).
__global__ void support_box_kernel(DevState* __restrict__ st, int mode, int nx, int ny, int nz, int z_lo,
                                   int z_hi, int* __restrict__ box) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    int lo = st->bbox_min[1][a], hi = st->bbox_max[1][a];
    if (mode == 0) {
      lo = min(lo, st->bbox_min[0][a]);
      hi = max(hi, st->bbox_max[0][a]);
    }
    lo = max(lo, 0);
    hi = min(hi, n[a] - 1);
    box[6 + 2 * a] = lo;
    box[6 + 2 * a + 1] = hi;
    if (a == 2) {
      lo = max(lo, z_lo);
      hi = min(hi, z_hi);
    }
    box[2 * a] = lo;
    box[2 * a + 1] = hi;
  }
  // the planes the field's preparation rewrites: the box's (the field of
  // this catalog is zero outside them) and those where the field buffer may
  // still be nonzero (every plane while that is unknown); afterwards the
  // field is zero outside the box's planes.  Computed again after the
  // preparation, with the same box, it leaves the record as it is.
  const int bz0 = box[10], bz1 = box[11];
  int r0 = bz0, r1 = bz1;
  if (!st->field_known) {
    r0 = 0;
    r1 = nz - 1;
  } else if (st->field_z0 <= st->field_z1) {
    r0 = r0 <= r1 ? min(r0, st->field_z0) : st->field_z0;
    r1 = bz0 <= bz1 ? max(r1, st->field_z1) : st->field_z1;
  }
  box[12] = r0;
  box[13] = r1;
  st->field_known = 1;
  st->field_z0 = bz0;
  st->field_z1 = bz1;
}

void launch_support_box(const Plan& p, int mode, cudaStream_t st) {
  const int z_lo = p.region ? p.region_z0 : 0;
  const int z_hi = p.region ? p.region_z1 - 1 : p.grid.n[2] - 1;
  support_box_kernel<<<1, 32, 0, st>>>(p.dstate, mode, p.grid.n[0], p.grid.n[1], p.grid.n[2], z_lo, z_hi, p.support);
}

cudaError_t launch_clear_counts(const Plan& p, int which, cudaStream_t st) {
  const int64_t plane = (int64_t)p.grid.n[0] * p.grid.n[1];
  clear_counts_kernel<<<elementwise_blocks(p, p.nc), 256, 0, st>>>(p.dstate, which, p.counts[which], plane,
                                                                   p.grid.n[2]);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(&p.dstate->counts_known[which], 1, sizeof(int), st);  // nonzero: known
}

void launch_prepare_randoms(const Plan& p, cudaStream_t st) {
  launch_support_box(p, 1, st);
  const int64_t plane = (int64_t)p.grid.n[0] * p.grid.n[1];
  ProfScope ps(p, ST_PREP, 0.0, 0.0, 8.0 * (double)plane, p.support + 6, st);
  prepare_randoms_kernel<<<elementwise_blocks(p, p.nc), 256, 0, st>>>(p.counts[1], p.field, p.support + 12, plane,
                                                                      p.dstate);
}

}  // namespace ck
