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
__global__ void sky_scan_kernel(Cosmo C, const double* __restrict__ seg, double* __restrict__ r) {
  double acc = 0.0;
  r[0] = 0.0;
  for (int k = 0; k < SK_NT; ++k) {
    acc += seg[k];
    r[k + 1] = C.dh * acc;
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

}  // namespace

}  // namespace ck

using namespace ck;

extern "C" ck_status ck_sky_to_cartesian(const ck_cosmology* cosmo, const float* ra_deg, const float* dec_deg,
                                         const float* redshift, int64_t n, float* x, float* y, float* z,
                                         void* stream) {
  if (!cosmo) return CK_ERR_BAD_POINTER;
  if (n < 0) return CK_ERR_ARG;
  const double vals[6] = {cosmo->h0, cosmo->omega_m, cosmo->omega_k, cosmo->omega_l, cosmo->c, cosmo->z_max};
  for (double v : vals)
    if (!isfinite(v)) return CK_ERR_ARG;
  if (!(cosmo->h0 > 0.0) || !(cosmo->c > 0.0) || !(cosmo->z_max > 0.0)) return CK_ERR_ARG;
  // E^2 > 0 over [0, z_max] (checked at the table nodes)
  for (int k = 0; k <= SK_NT; ++k) {
    const double a = 1.0 + cosmo->z_max * k / SK_NT;
    if (!(cosmo->omega_m * a * a * a + cosmo->omega_k * a * a + cosmo->omega_l > 0.0)) return CK_ERR_ARG;
  }
  if (n == 0) return CK_OK;
  if (!ra_deg || !dec_deg || !redshift || !x || !y || !z) return CK_ERR_BAD_POINTER;
  const void* ptrs[6] = {ra_deg, dec_deg, redshift, x, y, z};
  for (const void* q : ptrs)
    if (!is_device_ptr(q)) return CK_ERR_BAD_POINTER;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Cosmo C;
  C.om = cosmo->omega_m;
  C.ok = cosmo->omega_k;
  C.ol = cosmo->omega_l;
  C.dh = cosmo->c / cosmo->h0;
  C.h = cosmo->z_max / SK_NT;
  C.zmax = cosmo->z_max;
  double* tab = nullptr;  // seg[SK_NT] | r[SK_NT + 1] | dr[SK_NT + 1]
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tab), (size_t)(3 * SK_NT + 2) * sizeof(double), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CK_ERR_OOM;
  }
  double* seg = tab;
  double* r = seg + SK_NT;
  double* dr = r + SK_NT + 1;
  sky_table_kernel<<<(SK_NT + 1 + 255) / 256, 256, 0, st>>>(C, gauss_legendre(), seg, dr);
  sky_scan_kernel<<<1, 1, 0, st>>>(C, seg, r);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  sky_points_kernel<<<(unsigned)blocks, 256, 0, st>>>(C, r, dr, ra_deg, dec_deg, redshift, n, x, y, z);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(tab, st);
  return cuda_status(e != cudaSuccess ? e : f);
}
