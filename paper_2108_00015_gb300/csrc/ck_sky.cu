// ck_sky.cu -- survey coordinates to the grid's Cartesian frame (Sec. 2.2):
// the comoving distance of Eq. 3,
//   r(z) = (c / H0) int_0^z dz' / E(z'),  E^2 = O_M (1+z)^3 + O_k (1+z)^2 + O_L,
// and Eqs. 4-6, X = r cos(dec) cos(ra), Y = r cos(dec) sin(ra), Z = r sin(dec).
//  * sky_table_kernel: r(z) on SK_NT + 1 equally spaced nodes of [0, z_max]:
//    each thread integrates one interval by 8-point Gauss-Legendre
//    quadrature (FP64; the nodes and weights come from the host);
//  * sky_scan_kernel: one block forms the cumulative sums in a fixed order
//    (runs per thread, then shuffle scans), the same table from run to run;
//  * sky_points_kernel: per point, r(z) by cubic Hermite interpolation
//    between the two nodes around z (values and exact derivatives
//    c / (H0 E)), then the angles (degrees, sincospi in FP64); float32
//    outputs.  A redshift outside [0, z_max] or a non-finite input gives NaN
//    coordinates, which the gridding drops and counts.
// With SK_NT = 4096 the interpolation error is below 1e-12 of r for
// z_max <= 10, far below float32 rounding.
// The factorised randoms of Eq. 7 use the same table the other way round,
// R = N_tot P_ang(ra, dec) P_z(z) (dz/dr) g^3 / r^2 per cell of the box.
// FP64 runs at a small fraction of the float32 rate on this GPU, so:
//  * factorised_tables_kernel: z(r) and dz/dr on FR_NR + 1 nodes in r (z by
//    bisection of the distance table and Newton steps on its Hermite
//    interpolant, FP64), the cell centres per axis, N_tot g^3 P_ang and P_z,
//    all rounded to float32;
//  * factorised_fast_kernel: per cell in float32 (z and dz/dr by linear
//    interpolation in r, the angles by atan2f); a cell whose r, z or angle
//    lies within a margin of a decision edge (r(z_max), z_lo, z_hi, a bin
//    edge) larger than the float32 error bound is marked and queued instead;
//  * factorised_slow_kernel: the queued cells (or, if the queue overflowed,
//    every marked cell) by the FP64 path (cell_value_fp64), whose decisions
//    follow a plain FP64 evaluation's operation order, so every bin decision
//    is the FP64 one;
//  * factorised_reduce_kernel + factorised_total_kernel: the field's total,
//    nonzero cells and bounding box from the stored cells, per block in a
//    fixed order, then the blocks in order (the same total every run).
// Values: float32 cells within 13 float32 roundings (8e-7 relative) of the
// FP64 definition; FP64-path cells within one rounding.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {

namespace {

constexpr int SK_NT = 4096;  // table intervals
constexpr int SK_GL = 8;     // Gauss-Legendre points per interval

struct GaussLegendre {
  double x[SK_GL];  // nodes on [-1, 1]
  double w[SK_GL];
};

// Nodes: roots of the Legendre polynomial P_m by Newton's method from
// cosine initial guesses, with P_m and P_{m-1} from Bonnet's recurrence
// (k + 1) P_{k+1} = (2k + 1) x P_k - k P_{k-1}; weights 2 / ((1 - x^2) P_m'(x)^2).
GaussLegendre gauss_legendre() {
  GaussLegendre g;
  const int m = SK_GL;
  for (int i = 0; i < m; ++i) {
    double x = cos(M_PI * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;  // P_0, P_1
      for (int k = 1; k < m; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = m * (x * p1 - p0) / (x * x - 1.0);  // P_m'(x)
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    g.x[i] = x;
    g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return g;
}

struct Cosmo {
  double om, ok, ol;
  double dh;    // c / H0
  double h;     // table spacing in z
  double zmax;
};

__device__ __forceinline__ double inv_e(const Cosmo& C, double z) {
  const double a = 1.0 + z;
  return 1.0 / sqrt(C.om * a * a * a + C.ok * a * a + C.ol);
}

// seg[k] = int over [k h, (k + 1) h] of dz / E(z), k < SK_NT; dr[k] = c / (H0 E(k h)), k <= SK_NT
__global__ void sky_table_kernel(Cosmo C, GaussLegendre g, double* __restrict__ seg, double* __restrict__ dr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > SK_NT) return;
  dr[k] = C.dh * inv_e(C, k * C.h);
  if (k == SK_NT) return;
  const double mid = (k + 0.5) * C.h, half = 0.5 * C.h;
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < SK_GL; ++i) s += g.w[i] * inv_e(C, mid + half * g.x[i]);
  seg[k] = s * half;
}

// r[k] = c / H0 * (seg[0] + .. + seg[k - 1]), added in order by one thread
// r[k] = c / H0 * (seg[0] + .. + seg[k - 1]) by one block: each thread adds
// its SK_NT / 1024 segments in order, then shuffle scans within and across
// warps (a fixed order of additions: the same table from run to run).
constexpr int SK_SCAN = 1024;
static_assert(SK_NT % SK_SCAN == 0, "scan block");
__global__ void __launch_bounds__(SK_SCAN) sky_scan_kernel(Cosmo C, const double* __restrict__ seg,
                                                           double* __restrict__ r) {
  constexpr int PER = SK_NT / SK_SCAN;
  __shared__ double wtot[SK_SCAN / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  double v[PER];
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    s += seg[t * PER + j];
    v[j] = s;
  }
  double x = s;  // inclusive scan over the warp
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wtot[w] = x;
  __syncthreads();
  if (w == 0) {
    double y = wtot[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double q = __shfl_up_sync(0xFFFFFFFFu, y, off);
      if (lane >= off) y += q;
    }
    wtot[lane] = y;  // inclusive over warps
  }
  __syncthreads();
  double before = __shfl_up_sync(0xFFFFFFFFu, x, 1);
  if (lane == 0) before = 0.0;
  if (w > 0) before += wtot[w - 1];
  if (t == 0) r[0] = 0.0;
#pragma unroll
  for (int j = 0; j < PER; ++j) r[t * PER + j + 1] = C.dh * (before + v[j]);
}

struct Selection {
  const double* pang;  // [n_dec][n_ra]
  const double* pz;    // [n_z]
  int nra, ndec, nz;
  double zlo, zhi, ntot;
  double h0, c;
};

struct Box {
  int n[3];    // the caller's box
  int dim[3];  // the stored grid (the box, or its zero-padded transform grid)
  double o[3];
  double g, g3;
};

// z with H(z) = rr, H the cubic Hermite interpolant of the table, for
// 0 < rr <= r[SK_NT]: the interval by bisection of the nodes, then Newton
// steps in u from the linear estimate (H is monotone: r' = c / (H0 E) > 0).
__device__ __forceinline__ double z_of_r(const Cosmo& C, const double* __restrict__ r,
                                         const double* __restrict__ dr, double rr) {
  int lo = 0, hi = SK_NT;  // r[lo] < rr <= r[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(r + mid) < rr) lo = mid;
    else hi = mid;
  }
  const double r0 = __ldg(r + lo), r1 = __ldg(r + lo + 1);
  const double d0 = C.h * __ldg(dr + lo), d1 = C.h * __ldg(dr + lo + 1);
  double u = (rr - r0) / (r1 - r0);
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const double v = 1.0 - u;
    const double H = (1.0 + 2.0 * u) * v * v * r0 + u * v * v * d0 + u * u * (3.0 - 2.0 * u) * r1 - u * u * v * d1;
    const double dH = 6.0 * u * v * (r1 - r0) + v * (1.0 - 3.0 * u) * d0 + u * (3.0 * u - 2.0) * d1;
    u = fmin(fmax(u - (H - rr) / dH, 0.0), 1.0);
  }
  return (lo + u) * C.h;
}

constexpr int FR_THREADS = 256;
constexpr int FR_NR = 8192;  // intervals of the z(r), dz/dr tables on [0, r(z_max)]

// Eq. 7 at one cell in FP64: the exact path.  Every decision (r <= r(z_max),
// the redshift, right-ascension and declination bins) and the value follow
// the operation order of a plain FP64 evaluation.
__device__ double cell_value_fp64(const Cosmo& C, const double* __restrict__ r, const double* __restrict__ dr,
                                  const Selection& S, const Box& B, int ix, int iy, int iz) {
  const double kDeg = 180.0 / M_PI;
  const double X = __dadd_rn(B.o[0], __dmul_rn(ix + 0.5, B.g));
  const double Y = __dadd_rn(B.o[1], __dmul_rn(iy + 0.5, B.g));
  const double Z = __dadd_rn(B.o[2], __dmul_rn(iz + 0.5, B.g));
  const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y)), __dmul_rn(Z, Z)));
  if (!(rr > 0.0 && rr <= __ldg(r + SK_NT))) return 0.0;
  const double z = z_of_r(C, r, dr, rr);
  if (!(z >= S.zlo && z < S.zhi)) return 0.0;
  double ra = fmod(__dmul_rn(atan2(Y, X), kDeg), 360.0);
  if (ra < 0.0) ra += 360.0;
  const double dec = __dmul_rn(asin(__ddiv_rn(Z, rr)), kDeg);
  // bins (truncation toward zero; clamped into the tables)
  const int ia = max(0, min((int)__dmul_rn(__ddiv_rn(ra, 360.0), (double)S.nra), S.nra - 1));
  const int id = max(0, min((int)__dmul_rn(__ddiv_rn(__dadd_rn(dec, 90.0), 180.0), (double)S.ndec), S.ndec - 1));
  const int kz =
      max(0, min((int)__dmul_rn(__ddiv_rn(__dsub_rn(z, S.zlo), __dsub_rn(S.zhi, S.zlo)), (double)S.nz), S.nz - 1));
  const double a = 1.0 + z;
  const double dzdr = S.h0 * sqrt(C.om * a * a * a + C.ok * a * a + C.ol) / S.c;
  return S.ntot * __ldg(S.pang + (int64_t)id * S.nra + ia) * __ldg(S.pz + kz) * dzdr * B.g3 / (rr * rr);
}

// Float32 tables of the fast path (built by factorised_tables_kernel).
struct FastTabs {
  const float* zr;   // [FR_NR + 1] z at r_k = k r(z_max) / FR_NR
  const float* dzr;  // [FR_NR + 1] dz/dr = H0 E(z) / c at r_k
  const float* A;    // [n_dec * n_ra] N_tot g^3 P_ang
  const float* rmax;  // [2] r(z_max) and FR_NR / r(z_max)
  const float* pz;   // [n_z] P_z
  const float* ctr[3];  // cell centres per axis, FP64 values rounded to float32
  float ra_scale, dec_scale, z_scale;  // n_ra / 2 pi, n_dec / pi, n_z / (z_hi - z_lo)
  float zlo, zhi;
  float mz;                            // redshift margin of the fast decisions
  float tol_z, tol_ra, tol_dec;        // the margins in bin units
  float nra_f;
};

// Margins of the float32 decisions, about three times the float32 error
// bounds (each coordinate within 2^-24 relative of its FP64 value): r within
// 2.7e-7 relative (squares, two fused adds, the square root, r(z_max)'s
// rounding); the angles within 1.6e-6 rad (atan2f within 3 ulp, input
// rounding 2.4e-7 rad, the scale and its product, the wrap by n_ra); z
// within 9e-7 z_max (the r and scale errors times r z'/z <= 1.6, table
// and interpolation rounding, the bin scaling; linear interpolation on
// FR_NR intervals adds < 1e-8).  A cell closer than its margin to a
// decision edge takes the FP64 path.
// Cells left for the FP64 kernel hold this NaN pattern until it runs.
constexpr uint32_t kSlowMark = 0x7FC0DEADu;

constexpr float FR_MR = 2e-6f;    // relative, r against r(z_max) (error bound 2.7e-7)
constexpr float FR_MANG = 5e-6f;  // radians (error bound 1.6e-6)
// (the redshift margin, 3e-6 z_max against a bound of 9e-7 z_max, is FastTabs::mz)

__global__ void factorised_tables_kernel(Cosmo C, const double* __restrict__ r, const double* __restrict__ dr,
                                         Selection S, Box B, double h0, double c, float* __restrict__ zr,
                                         float* __restrict__ dzr, float* __restrict__ A, float* __restrict__ pzf,
                                         float* __restrict__ cx, float* __restrict__ cy, float* __restrict__ cz,
                                         float* __restrict__ rmax_f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const double rmax = r[SK_NT];
  if (t == 0) {
    rmax_f[0] = (float)rmax;
    rmax_f[1] = (float)(FR_NR / rmax);
  }
  for (int k = t; k <= FR_NR; k += stride) {
    const double rk = rmax * k / FR_NR;
    const double z = k == 0 ? 0.0 : (k == FR_NR ? C.zmax : z_of_r(C, r, dr, rk));
    const double a = 1.0 + z;
    zr[k] = (float)z;
    dzr[k] = (float)(h0 * sqrt(C.om * a * a * a + C.ok * a * a + C.ol) / c);
  }
  const int na = S.nra * S.ndec;
  for (int k = t; k < na; k += stride) A[k] = (float)(S.ntot * B.g3 * S.pang[k]);
  for (int k = t; k < S.nz; k += stride) pzf[k] = (float)S.pz[k];
  for (int k = t; k < B.n[0]; k += stride) cx[k] = (float)__dadd_rn(B.o[0], __dmul_rn(k + 0.5, B.g));
  for (int k = t; k < B.n[1]; k += stride) cy[k] = (float)__dadd_rn(B.o[1], __dmul_rn(k + 0.5, B.g));
  for (int k = t; k < B.n[2]; k += stride) cz[k] = (float)__dadd_rn(B.o[2], __dmul_rn(k + 0.5, B.g));
}

// The rows (iy, iz) of warp w: w, w + W, w + 2W, ... with (iy, iz) advanced
// by carries instead of a division per row (integer division converts
// through floating point).
struct RowWalk {
  unsigned row, nrows, step;
  int iy, iz, n1, sy, sz;  // step = sz n1 + sy
  __device__ RowWalk(unsigned first, unsigned stride, int ny, int nz) : row(first), step(stride), n1(ny) {
    nrows = (unsigned)ny * (unsigned)nz;
    iy = (int)(first % (unsigned)ny);
    iz = (int)(first / (unsigned)ny);
    sy = (int)(stride % (unsigned)ny);
    sz = (int)(stride / (unsigned)ny);
  }
  __device__ bool ok() const { return row < nrows; }
  __device__ void next() {
    row += step;
    iy += sy;
    iz += sz;
    if (iy >= n1) {
      iy -= n1;
      ++iz;
    }
  }
};

// floor(t) for 0 <= t < 2^22 without a conversion instruction: t + 2^23
// rounded down holds floor(t) in its low mantissa bits.  Also returns
// whether t lies within tol of an integer (a bin edge).
__device__ __forceinline__ int bin_of(float t, float tol, bool* near) {
  const float b = __fadd_rd(t, 8388608.0f);
  const float f = t - (b - 8388608.0f);
  *near = fminf(f, 1.0f - f) <= tol;
  return __float_as_int(b) - 0x4B000000;
}

// Per cell of the box: Eq. 7 in float32 where every decision is clear of
// its edge by the margins above; otherwise the cell goes to the FP64 queue
// (or, when the queue is full, the FP64 path in place).
__global__ void __launch_bounds__(FR_THREADS) factorised_fast_kernel(
    Cosmo C, const double* __restrict__ r, const double* __restrict__ dr, Selection S, Box B, FastTabs T,
    uint32_t* __restrict__ cells, uint32_t* __restrict__ queue, unsigned int* __restrict__ qn, unsigned int qcap) {
  const float half_pi = 1.57079632679489661923f;
  const float rmax = __ldg(T.rmax), inv_h = __ldg(T.rmax + 1);
  // one warp per row of cells (iy, iz), lanes along x; 32-bit index
  // arithmetic (box axes <= 512; a 64-bit division would use the FP64 pipe)
  const unsigned lane = threadIdx.x & 31u;
  for (RowWalk w(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), gridDim.x * (blockDim.x >> 5), B.n[1], B.n[2]);
       w.ok(); w.next()) {
    const unsigned row = w.row;
    const int iy = w.iy, iz = w.iz;
    const float Y = __ldg(T.ctr[1] + iy), Z = __ldg(T.ctr[2] + iz);
    uint32_t* __restrict__ crow = cells + ((int64_t)iz * B.dim[1] + iy) * B.dim[0];
    for (int ix = lane; ix < B.n[0]; ix += 32) {
      const unsigned i = row * (unsigned)B.n[0] + (unsigned)ix;
      const float X = __ldg(T.ctr[0] + ix);
      const float rho2 = fmaf(X, X, Y * Y);
      const float r2 = fmaf(Z, Z, rho2);
      const float rf = sqrtf(r2);
      float v = 0.0f;
      bool slow = false;
      if (r2 == 0.0f || fabsf(rf - rmax) <= FR_MR * rmax) {
        slow = true;
      } else if (rf < rmax) {
        // rf < rmax (1 - FR_MR): u < FR_NR
        float u = rf * inv_h;
        bool unused;
        const int k = min(bin_of(u, 0.0f, &unused), FR_NR - 1);
        u -= __int_as_float(0x4B000000 + k) - 8388608.0f;
        const float z0 = __ldg(T.zr + k), z1 = __ldg(T.zr + k + 1);
        const float zf = fmaf(u, z1 - z0, z0);
        if (fabsf(zf - T.zlo) <= T.mz || fabsf(zf - T.zhi) <= T.mz) {
          slow = true;
        } else if (zf > T.zlo && zf < T.zhi) {
          // bin coordinates, clamped at 0 (the lower edge of bin 0 decides nothing)
          const float tz = fmaxf((zf - T.zlo) * T.z_scale, 0.0f);
          float ta = atan2f(Y, X) * T.ra_scale;
          if (ta < 0.0f) ta += T.nra_f;
          const float td = fmaxf((atan2f(Z, sqrtf(rho2)) + half_pi) * T.dec_scale, 0.0f);
          bool nz_, na_, nd_;
          const int kz = min(bin_of(tz, T.tol_z, &nz_), S.nz - 1);
          const int ia = min(bin_of(fmaxf(ta, 0.0f), T.tol_ra, &na_), S.nra - 1);
          const int id = min(bin_of(td, T.tol_dec, &nd_), S.ndec - 1);
          if (nz_ || na_ || nd_) {
            slow = true;
          } else {
            const float d0 = __ldg(T.dzr + k), d1 = __ldg(T.dzr + k + 1);
            const float dzdr = fmaf(u, d1 - d0, d0);
            v = __ldg(T.A + id * S.nra + ia) * __ldg(T.pz + kz) * dzdr * __frcp_rn(r2);
          }
        }
      }
      uint32_t out = __float_as_uint(v);
      if (slow) {
        // the FP64 kernel writes this cell: from the queue, or (queue full)
        // by finding the mark
        const unsigned int q = atomicAdd(qn, 1u);
        if (q < qcap) queue[q] = i;
        out = kSlowMark;
      }
      crow[ix] = out;
    }
  }
}

// The queued cells in FP64, in full warps; if the queue overflowed, also
// every cell still holding the mark.
__global__ void __launch_bounds__(FR_THREADS) factorised_slow_kernel(
    Cosmo C, const double* __restrict__ r, const double* __restrict__ dr, Selection S, Box B,
    uint32_t* __restrict__ cells, const uint32_t* __restrict__ queue, const unsigned int* __restrict__ qn,
    unsigned int qcap) {
  const unsigned int total = *qn;
  if (total > qcap) {
    for (RowWalk w(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), gridDim.x * (blockDim.x >> 5), B.n[1],
                   B.n[2]);
         w.ok(); w.next()) {
      uint32_t* __restrict__ crow = cells + ((int64_t)w.iz * B.dim[1] + w.iy) * B.dim[0];
      for (int ix = threadIdx.x & 31; ix < B.n[0]; ix += 32)
        if (crow[ix] == kSlowMark) crow[ix] = __float_as_uint((float)cell_value_fp64(C, r, dr, S, B, ix, w.iy, w.iz));
    }
    return;  // the queued cells hold the mark too
  }
  const unsigned int n = total;
  for (unsigned int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const unsigned i = queue[j];
    const int ix = (int)(i % (unsigned)B.n[0]);
    const unsigned t = i / (unsigned)B.n[0];
    const int iy = (int)(t % (unsigned)B.n[1]);
    const int iz = (int)(t / (unsigned)B.n[1]);
    const float v = (float)cell_value_fp64(C, r, dr, S, B, ix, iy, iz);
    cells[((int64_t)iz * B.dim[1] + iy) * B.dim[0] + ix] = __float_as_uint(v);
  }
}

// The field's totals from its stored cells: per block the FP64 sum (a fixed
// shuffle tree, then the warps in order), the nonzero cells and their
// bounding box.
__global__ void __launch_bounds__(FR_THREADS) factorised_reduce_kernel(Box B, const uint32_t* __restrict__ cells,
                                                                      double* __restrict__ part, DevState* st) {
  double sum = 0.0;
  unsigned long long kept = 0;
  int bmin[3] = {INT_MAX, INT_MAX, INT_MAX}, bmax[3] = {INT_MIN, INT_MIN, INT_MIN};
  const int lane = threadIdx.x & 31;
  const bool vec = (B.n[0] & 3) == 0 && (B.dim[0] & 3) == 0;  // rows start on 16-byte boundaries
  // per lane: a compensated float32 sum (TwoSum: hi + lo carries the
  // rounding error of every addition), converted to FP64 once at the end
  float hi = 0.0f, lo = 0.0f;
  for (RowWalk w(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), gridDim.x * (blockDim.x >> 5), B.n[1], B.n[2]);
       w.ok(); w.next()) {
    const int iy = w.iy, iz = w.iz;
    const uint32_t* __restrict__ crow = cells + ((int64_t)iz * B.dim[1] + iy) * B.dim[0];
    auto take = [&](float v, int ix) {
      if (v != 0.0f) {
        ++kept;
        const float s2 = hi + v;
        const float bp = s2 - hi;
        lo += (hi - (s2 - bp)) + (v - bp);
        hi = s2;
        bmin[0] = min(bmin[0], ix); bmax[0] = max(bmax[0], ix);
        bmin[1] = min(bmin[1], iy); bmax[1] = max(bmax[1], iy);
        bmin[2] = min(bmin[2], iz); bmax[2] = max(bmax[2], iz);
      }
    };
    if (vec) {
      // 16-byte loads, four in flight per lane
      const float4* __restrict__ c4 = reinterpret_cast<const float4*>(crow);
      const int nv = B.n[0] >> 2;
      for (int b0 = 0; b0 < nv; b0 += 128) {
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = b0 + u * 32 + lane;
          q[u] = j < nv ? __ldg(c4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int ix = 4 * (b0 + u * 32 + lane);
          take(q[u].x, ix);
          take(q[u].y, ix + 1);
          take(q[u].z, ix + 2);
          take(q[u].w, ix + 3);
        }
      }
    } else {
      for (int ix = lane; ix < B.n[0]; ix += 32) take(__uint_as_float(__ldg(crow + ix)), ix);
    }
  }
  sum = (double)hi + (double)lo;
  // block reduction: a fixed shuffle tree, then the warps in order
  for (int off = 16; off > 0; off >>= 1) {
    sum += __shfl_down_sync(0xFFFFFFFFu, sum, off);
    kept += __shfl_down_sync(0xFFFFFFFFu, kept, off);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bmin[a] = __reduce_min_sync(0xFFFFFFFFu, bmin[a]);
    bmax[a] = __reduce_max_sync(0xFFFFFFFFu, bmax[a]);
  }
  __shared__ double ssum[FR_THREADS / 32];
  __shared__ unsigned long long skept[FR_THREADS / 32];
  __shared__ int smin[FR_THREADS / 32][3], smax[FR_THREADS / 32][3];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ssum[w] = sum;
    skept[w] = kept;
    for (int a = 0; a < 3; ++a) { smin[w][a] = bmin[a]; smax[w][a] = bmax[a]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S2 = 0.0;
    unsigned long long K = 0;
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int j = 0; j < FR_THREADS / 32; ++j) {
      S2 += ssum[j];
      K += skept[j];
      for (int a = 0; a < 3; ++a) { mn[a] = min(mn[a], smin[j][a]); mx[a] = max(mx[a], smax[j][a]); }
    }
    part[blockIdx.x] = S2;
    if (K) {
      atomicAdd(&st->kept[1], K);
      for (int a = 0; a < 3; ++a) {
        atomicMin(&st->bbox_min[1][a], mn[a]);
        atomicMax(&st->bbox_max[1][a], mx[a]);
      }
    }
  }
}

// One warp: lane j adds blocks j, j + 32, .. in order, then a fixed xor tree.
__global__ void factorised_total_kernel(const double* __restrict__ part, int nblocks, DevState* st) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += part[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if (lane == 0) {
    st->fsum[1] = s;
    st->weighted[1] = 2;
  }
}

__global__ void sky_points_kernel(Cosmo C, const double* __restrict__ r, const double* __restrict__ dr,
                                  const float* __restrict__ ra, const float* __restrict__ dec,
                                  const float* __restrict__ zs, int64_t n, float* __restrict__ X,
                                  float* __restrict__ Y, float* __restrict__ Z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double z = zs[i], a = ra[i], d = dec[i];
    if (!(z >= 0.0 && z <= C.zmax) || !isfinite(a) || !isfinite(d)) {
      X[i] = Y[i] = Z[i] = __int_as_float(0x7fc00000);
      continue;
    }
    const double t = z / C.h;
    const int k = min((int)t, SK_NT - 1);
    const double u = t - k, v = 1.0 - u;
    // cubic Hermite: values r_k, r_{k+1}, derivatives (per unit u) h dr
    const double rr = (1.0 + 2.0 * u) * v * v * r[k] + u * v * v * C.h * dr[k] + u * u * (3.0 - 2.0 * u) * r[k + 1] -
                      u * u * v * C.h * dr[k + 1];
    double sa, ca, sd, cd;
    sincospi(a / 180.0, &sa, &ca);
    sincospi(d / 180.0, &sd, &cd);
    X[i] = (float)(rr * cd * ca);
    Y[i] = (float)(rr * cd * sa);
    Z[i] = (float)(rr * sd);
  }
}

// Validation shared by both entry points: finite parameters, h0, c,
// z_max > 0 and E^2 > 0 over [0, z_max] (checked at the table nodes).
ck_status check_cosmology(const ck_cosmology* cosmo) {
  if (!cosmo) return CK_ERR_BAD_POINTER;
  const double vals[6] = {cosmo->h0, cosmo->omega_m, cosmo->omega_k, cosmo->omega_l, cosmo->c, cosmo->z_max};
  for (double v : vals)
    if (!isfinite(v)) return CK_ERR_ARG;
  if (!(cosmo->h0 > 0.0) || !(cosmo->c > 0.0) || !(cosmo->z_max > 0.0)) return CK_ERR_ARG;
  for (int k = 0; k <= SK_NT; ++k) {
    const double a = 1.0 + cosmo->z_max * k / SK_NT;
    if (!(cosmo->omega_m * a * a * a + cosmo->omega_k * a * a + cosmo->omega_l > 0.0)) return CK_ERR_ARG;
  }
  return CK_OK;
}

Cosmo make_cosmo(const ck_cosmology* cosmo) {
  Cosmo C;
  C.om = cosmo->omega_m;
  C.ok = cosmo->omega_k;
  C.ol = cosmo->omega_l;
  C.dh = cosmo->c / cosmo->h0;
  C.h = cosmo->z_max / SK_NT;
  C.zmax = cosmo->z_max;
  return C;
}

// The distance table r[SK_NT + 1] and its derivatives dr[SK_NT + 1] in
// tab (3 SK_NT + 2 doubles: seg | r | dr).
void launch_table(const Cosmo& C, double* tab, cudaStream_t st) {
  double* seg = tab;
  double* r = seg + SK_NT;
  double* dr = r + SK_NT + 1;
  sky_table_kernel<<<(SK_NT + 1 + 255) / 256, 256, 0, st>>>(C, gauss_legendre(), seg, dr);
  sky_scan_kernel<<<1, SK_SCAN, 0, st>>>(C, seg, r);
}

int device_sms() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

ck_status check_factorised(const ck_cosmology* cosmo, const ck_selection* sel) {
  const ck_status cs = check_cosmology(cosmo);
  if (cs != CK_OK) return cs;
  if (!sel || !sel->p_ang || !sel->p_z) return CK_ERR_BAD_POINTER;
  // the tables are read here on the host: device memory is refused first
  if (is_device_ptr(sel->p_ang) || is_device_ptr(sel->p_z)) return CK_ERR_BAD_POINTER;
  if (sel->n_ra < 1 || sel->n_dec < 1 || sel->n_z < 1) return CK_ERR_ARG;
  if (sel->n_ra > (1 << 20) || sel->n_dec > (1 << 20) || sel->n_z > (1 << 20)) return CK_ERR_ARG;
  if ((int64_t)sel->n_ra * sel->n_dec > ((int64_t)1 << 26)) return CK_ERR_ARG;
  if (!isfinite(sel->n_tot) || !(sel->n_tot >= 0.0)) return CK_ERR_ARG;
  if (!isfinite(sel->z_lo) || !isfinite(sel->z_hi) || !(sel->z_lo >= 0.0) || !(sel->z_hi > sel->z_lo))
    return CK_ERR_ARG;
  const int64_t na = (int64_t)sel->n_ra * sel->n_dec;
  for (int64_t i = 0; i < na; ++i)
    if (!isfinite(sel->p_ang[i]) || !(sel->p_ang[i] >= 0.0)) return CK_ERR_ARG;
  for (int i = 0; i < sel->n_z; ++i)
    if (!isfinite(sel->p_z[i]) || !(sel->p_z[i] >= 0.0)) return CK_ERR_ARG;
  return CK_OK;
}

ck_status launch_factorised_randoms(Plan& p, const ck_cosmology* cosmo, const ck_selection* sel,
                                    cudaStream_t st) {
  const Cosmo C = make_cosmo(cosmo);
  const int64_t na = (int64_t)sel->n_ra * sel->n_dec;
  const int64_t nbox = (int64_t)p.box_n[0] * p.box_n[1] * p.box_n[2];
  const int sms = device_sms();
  const int64_t nrows = (int64_t)p.box_n[1] * p.box_n[2];  // a warp per row of cells
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nrows + FR_THREADS / 32 - 1) / (FR_THREADS / 32),
                                                                 (int64_t)sms * 8));
  // FP64 queue for cells near a decision edge (indices into the box)
  // (1/64 of the box: near-edge cells are a small fraction on real selections;
  // beyond it the FP64 kernel finds the marked cells by a scan instead)
  const unsigned int qcap = (unsigned int)std::min<int64_t>(nbox / 64 + 64, (int64_t)1 << 22);
  // scratch: doubles (table seg | r | dr, p_ang, p_z, per-block sums), then
  // floats (z(r), dz/dr, A, P_z, centres), then the queue and its counter
  const size_t nd = (size_t)(3 * SK_NT + 2) + (size_t)na + (size_t)sel->n_z + (size_t)blocks;
  const size_t nf = 2 * (size_t)(FR_NR + 1) + (size_t)na + (size_t)sel->n_z + (size_t)p.box_n[0] + p.box_n[1] +
                    p.box_n[2] + 2;
  const size_t nf_pad = (nf + 3) / 4 * 4;
  const size_t bytes = nd * 8 + nf_pad * 4 + ((size_t)qcap + 4) * 4;
  unsigned char* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CK_ERR_OOM;
  }
  double* tab = reinterpret_cast<double*>(scratch);
  double* r = tab + SK_NT;
  double* dr = r + SK_NT + 1;
  double* pang = dr + SK_NT + 1;
  double* pz = pang + na;
  double* part = pz + sel->n_z;
  float* zr = reinterpret_cast<float*>(scratch + nd * 8);
  float* dzr = zr + FR_NR + 1;
  float* A = dzr + FR_NR + 1;
  float* pzf = A + na;
  float* cx = pzf + sel->n_z;
  float* cy = cx + p.box_n[0];
  float* cz = cy + p.box_n[1];
  float* rmf = cz + p.box_n[2];
  uint32_t* queue = reinterpret_cast<uint32_t*>(scratch + nd * 8 + nf_pad * 4);
  unsigned int* qn = queue + qcap;
  e = cudaMemcpyAsync(pang, sel->p_ang, (size_t)na * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pz, sel->p_z, (size_t)sel->n_z * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(qn, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    launch_table(C, tab, st);
    Selection S;
    S.pang = pang;
    S.pz = pz;
    S.nra = sel->n_ra;
    S.ndec = sel->n_dec;
    S.nz = sel->n_z;
    S.zlo = sel->z_lo;
    S.zhi = sel->z_hi;
    S.ntot = sel->n_tot;
    S.h0 = cosmo->h0;
    S.c = cosmo->c;
    Box B;
    for (int a = 0; a < 3; ++a) {
      B.n[a] = p.box_n[a];
      B.dim[a] = p.grid.n[a];
      B.o[a] = p.grid.origin[a];
    }
    B.g = p.grid.cell;
    B.g3 = p.grid.cell * p.grid.cell * p.grid.cell;
    factorised_tables_kernel<<<64, 256, 0, st>>>(C, r, dr, S, B, cosmo->h0, cosmo->c, zr, dzr, A, pzf, cx, cy, cz, rmf);
    // the scales of the float decisions (r(z_max) is read from the table on the device)
    FastTabs T;
    T.zr = zr;
    T.dzr = dzr;
    T.A = A;
    T.rmax = rmf;
    T.pz = pzf;
    T.ctr[0] = cx;
    T.ctr[1] = cy;
    T.ctr[2] = cz;
    const double two_pi = 2.0 * M_PI;
    T.ra_scale = (float)(sel->n_ra / two_pi);
    T.dec_scale = (float)(sel->n_dec / M_PI);
    T.z_scale = (float)(sel->n_z / (sel->z_hi - sel->z_lo));
    T.zlo = (float)sel->z_lo;
    T.zhi = (float)sel->z_hi;
    T.mz = (float)(3e-6 * cosmo->z_max);
    T.tol_z = (float)(3e-6 * cosmo->z_max * sel->n_z / (sel->z_hi - sel->z_lo));
    T.tol_ra = (float)(FR_MANG * sel->n_ra / two_pi);
    T.tol_dec = (float)(FR_MANG * sel->n_dec / M_PI);
    T.nra_f = (float)sel->n_ra;
    ProfScope ps(p, ST_SELECTION, 8.0 * (double)nbox, st);
    factorised_fast_kernel<<<blocks, FR_THREADS, 0, st>>>(C, r, dr, S, B, T, p.counts[1], queue, qn, qcap);
    factorised_slow_kernel<<<sms * 4, FR_THREADS, 0, st>>>(C, r, dr, S, B, p.counts[1], queue, qn, qcap);
    factorised_reduce_kernel<<<blocks, FR_THREADS, 0, st>>>(B, p.counts[1], part, p.dstate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    factorised_total_kernel<<<1, 32, 0, st>>>(part, blocks, p.dstate);
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(scratch, st);
  return cuda_status(e != cudaSuccess ? e : f);
}

}  // namespace ck

using namespace ck;

extern "C" ck_status ck_sky_to_cartesian(const ck_cosmology* cosmo, const float* ra_deg, const float* dec_deg,
                                         const float* redshift, int64_t n, float* x, float* y, float* z,
                                         void* stream) {
  if (!cosmo) return CK_ERR_BAD_POINTER;
  if (n < 0) return CK_ERR_ARG;
  const ck_status cs = check_cosmology(cosmo);
  if (cs != CK_OK) return cs;
  if (n == 0) return CK_OK;
  if (!ra_deg || !dec_deg || !redshift || !x || !y || !z) return CK_ERR_BAD_POINTER;
  const void* ptrs[6] = {ra_deg, dec_deg, redshift, x, y, z};
  for (const void* q : ptrs)
    if (!is_device_ptr(q)) return CK_ERR_BAD_POINTER;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Cosmo C = make_cosmo(cosmo);
  double* tab = nullptr;  // seg[SK_NT] | r[SK_NT + 1] | dr[SK_NT + 1]
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tab), (size_t)(3 * SK_NT + 2) * sizeof(double), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CK_ERR_OOM;
  }
  double* r = tab + SK_NT;
  double* dr = r + SK_NT + 1;
  launch_table(C, tab, st);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 8);
  sky_points_kernel<<<(unsigned)blocks, 256, 0, st>>>(C, r, dr, ra_deg, dec_deg, redshift, n, x, y, z);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(tab, st);
  return cuda_status(e != cudaSuccess ? e : f);
}
