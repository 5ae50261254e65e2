// ck_sky.cu -- survey coordinates to the grid's Cartesian frame (Sec. 2.1):
// the comoving distance of Eq. 3,
//   r(z) = (c / H0) int_0^z dz' / E(z'),  E^2 = O_M (1+z)^3 + O_k (1+z)^2 + O_L,
// and Eqs. 4-6, X = r cos(dec) cos(ra), Y = r cos(dec) sin(ra), Z = r sin(dec).
//  * sky_table_kernel: r(z) on SK_NT + 1 equally spaced nodes of [0, z_max]:
//    each thread integrates one interval by 8-point Gauss-Legendre
//    quadrature (FP64; the nodes and weights come from the host), one thread
//    then adds the intervals in order (the same table from run to run);
//  * sky_points_kernel: per point, r(z) by cubic Hermite interpolation
//    between the two nodes around z (values and exact derivatives
//    c / (H0 E)), then the angles (degrees, sincospi in FP64); float32
//    outputs.  A redshift outside [0, z_max] or a non-finite input gives NaN
//    coordinates, which the gridding drops and counts.
// With SK_NT = 4096 the interpolation error is below 1e-12 of r for
// z_max <= 10, far below float32 rounding.
// The factorised randoms of Eq. 7 use the same table the other way round:
//  * factorised_randoms_kernel: per cell of the plan's box, z(r) by a binary
//    search of the nodes and Newton steps on the Hermite interpolant, then
//    R = N_tot P_ang(ra, dec) P_z(z) (dz/dr) g^3 / r^2 in FP64, stored as
//    float32; the cell centre, r and the angle bins are evaluated in the
//    same operation order as a plain FP64 evaluation (no contraction), so
//    that the bin decisions are those of such an evaluation;
//  * factorised_total_kernel: the per-block FP64 partial sums added in
//    block order (the same total from run to run).
#include <math.h>

#include <limits.h>

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
__global__ void sky_scan_kernel(Cosmo C, const double* __restrict__ seg, double* __restrict__ r) {
  double acc = 0.0;
  r[0] = 0.0;
  for (int k = 0; k < SK_NT; ++k) {
    acc += seg[k];
    r[k + 1] = C.dh * acc;
  }
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

__global__ void __launch_bounds__(FR_THREADS) factorised_randoms_kernel(
    Cosmo C, const double* __restrict__ r, const double* __restrict__ dr, Selection S, Box B,
    uint32_t* __restrict__ cells, double* __restrict__ part, DevState* st) {
  const double kDeg = 180.0 / M_PI;
  const double rmax = __ldg(r + SK_NT);
  const int64_t nbox = (int64_t)B.n[0] * B.n[1] * B.n[2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double sum = 0.0;
  unsigned long long kept = 0;
  int bmin[3] = {INT_MAX, INT_MAX, INT_MAX}, bmax[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbox; i += stride) {
    const int ix = (int)(i % B.n[0]);
    const int64_t t = i / B.n[0];
    const int iy = (int)(t % B.n[1]);
    const int iz = (int)(t / B.n[1]);
    const double X = __dadd_rn(B.o[0], __dmul_rn(ix + 0.5, B.g));
    const double Y = __dadd_rn(B.o[1], __dmul_rn(iy + 0.5, B.g));
    const double Z = __dadd_rn(B.o[2], __dmul_rn(iz + 0.5, B.g));
    const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y)), __dmul_rn(Z, Z)));
    double v = 0.0;
    if (rr > 0.0 && rr <= rmax) {
      const double z = z_of_r(C, r, dr, rr);
      if (z >= S.zlo && z < S.zhi) {
        double ra = fmod(__dmul_rn(atan2(Y, X), kDeg), 360.0);
        if (ra < 0.0) ra += 360.0;
        const double dec = __dmul_rn(asin(__ddiv_rn(Z, rr)), kDeg);
        // bins (truncation toward zero; clamped into the tables)
        const int ia = max(0, min((int)__dmul_rn(__ddiv_rn(ra, 360.0), (double)S.nra), S.nra - 1));
        const int id =
            max(0, min((int)__dmul_rn(__ddiv_rn(__dadd_rn(dec, 90.0), 180.0), (double)S.ndec), S.ndec - 1));
        const int kz = max(
            0, min((int)__dmul_rn(__ddiv_rn(__dsub_rn(z, S.zlo), __dsub_rn(S.zhi, S.zlo)), (double)S.nz), S.nz - 1));
        const double a = 1.0 + z;
        const double dzdr = S.h0 * sqrt(C.om * a * a * a + C.ok * a * a + C.ol) / S.c;
        v = S.ntot * __ldg(S.pang + (int64_t)id * S.nra + ia) * __ldg(S.pz + kz) * dzdr * B.g3 / (rr * rr);
      }
    }
    cells[((int64_t)iz * B.dim[1] + iy) * B.dim[0] + ix] = __float_as_uint((float)v);
    if (v != 0.0) {
      ++kept;
      sum += v;
      bmin[0] = min(bmin[0], ix); bmax[0] = max(bmax[0], ix);
      bmin[1] = min(bmin[1], iy); bmax[1] = max(bmax[1], iy);
      bmin[2] = min(bmin[2], iz); bmax[2] = max(bmax[2], iz);
    }
  }
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

__global__ void factorised_total_kernel(const double* __restrict__ part, int nblocks, DevState* st) {
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[b];
  st->fsum[1] = s;
  st->weighted[1] = 2;
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
  sky_scan_kernel<<<1, 1, 0, st>>>(C, seg, r);
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
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nbox + FR_THREADS - 1) / FR_THREADS,
                                                                 (int64_t)device_sms() * 8));
  // scratch: table | p_ang | p_z | per-block sums
  const size_t nd = (size_t)(3 * SK_NT + 2) + (size_t)na + (size_t)sel->n_z + (size_t)blocks;
  double* tab = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tab), nd * sizeof(double), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CK_ERR_OOM;
  }
  double* r = tab + SK_NT;
  double* dr = r + SK_NT + 1;
  double* pang = dr + SK_NT + 1;
  double* pz = pang + na;
  double* part = pz + sel->n_z;
  e = cudaMemcpyAsync(pang, sel->p_ang, (size_t)na * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pz, sel->p_z, (size_t)sel->n_z * sizeof(double), cudaMemcpyHostToDevice, st);
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
    factorised_randoms_kernel<<<blocks, FR_THREADS, 0, st>>>(C, r, dr, S, B, p.counts[1], part, p.dstate);
    factorised_total_kernel<<<1, 1, 0, st>>>(part, blocks, p.dstate);
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(tab, st);
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
