// ck_fft.cu -- the convolution stage (Sec. 2.4, Eqs. 9-10) by FFT: the
// forward and inverse 3D transforms of a plan, with the kernel-spectrum
// multiply fused into the first inverse pass, and the once-per-plan build of
// the shell spectra K^_s.  The pass kernels are in ck_fft_core.cuh.
//
// Forward (one field): x pass (real rows -> half spectrum), y pass, z pass.
// Inverse (all shells of one field at once): one z pass that reads the
// spectrum once and writes spectrum * K^_s transformed along z for every
// shell, then one y pass and one x pass over all shells.  Plans whose shells
// reach few planes take the z step directly (ck_zconv.cu): the forward
// transform stops after the y pass and the direct filter replaces the K^ z
// pass.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ck_fft_core.cuh"

namespace ck {

using fft::KhatArgs;
using fft::StridedView;
using fft::kT;

ck_status fft_init_attributes() { return CK_OK; }

void launch_fft_forward(const Plan& p, const float* in, float2* spec, cudaStream_t st, const int* box, bool conv) {
  const int nx = p.grid.n[0], ny = p.grid.n[1], nz = p.grid.n[2];
  // the direct z step reads the spectrum untransformed along z
  const bool direct = conv && p.tune.z_direct && p.kz_dz > 0;
  if (conv) {
    p.spec_direct = direct;
    p.spec_in_box = box;
  }
  const int64_t rows = (int64_t)ny * nz;
  const double H = (double)nz * ny * (nx / 2 + 1);
  const double row = 8.0 * (nx / 2 + 1);  // bytes of one half-spectrum row
  // the field is zero outside the box: on 512-point y and z axes the x pass
  // transforms the box's rows, the y pass its planes (reading its rows) and
  // the z pass reads its planes; every output of the z pass is written
  if (ny != 512 || nz != 512) box = nullptr;
  {
    ProfScope ps(p, ST_FFT_X_R2C, box ? 0.0 : 4.0 * (double)p.nc + 8.0 * H, 4.0 * nx + row, 0.0, box, st);
    fft::launch_x_r2c(nx / 2, in, spec, nx, p.px, rows, p.fx_half, p.stw[0], p.tw[0], p.sm_count, st, box, ny);
  }
  {
    ProfScope ps(p, ST_FFT_Y_FWD, box ? 0.0 : 16.0 * H, row, row * ny, box, st);
    StridedView v{p.px, (int64_t)ny * p.px, p.px, nz};
    fft::launch_strided(ny, false, spec, spec, v, p.fy, p.stw[1], p.tw[1], p.tune.fwd_cols, p.sm_count, st, box, nz,
                        fft::kPrunePlanes | fft::kPruneInY);
  }
  if (!direct) {
    ProfScope ps(p, ST_FFT_Z_FWD, box ? 8.0 * H : 16.0 * H, 0.0, row * ny, box, st);
    StridedView v{(int64_t)ny * p.px, 0, ny * p.px, 1};
    fft::launch_strided(nz, false, spec, spec, v, p.fz, p.stw[2], p.tw[2], p.tune.fwd_cols, p.sm_count, st, box, nz,
                        fft::kPruneInZ);
  }
}

// Inverse z and y passes of nshells spectra: spec * K^_s for shells shell0 ..
// (shell0 >= 0) or spec itself (shell0 < 0, nshells == 1), into the scratch
// spectra tmp[s] (stride spec_elems).  The z step of a convolution of a
// spectrum left untransformed along z (p.spec_direct) is the direct filter.
void launch_inverse_zy(const Plan& p, const float2* spec, int shell0, int nshells, float2* tmp, cudaStream_t st,
                       const int* box) {
  const int nx = p.grid.n[0], ny = p.grid.n[1], nz = p.grid.n[2];
  const double H = (double)nz * ny * (nx / 2 + 1);
  const double row = 8.0 * (nx / 2 + 1);  // bytes of one half-spectrum row
  // support pruning on the 512-point register passes; the other lengths
  // transform and write every plane (the fused x pass visits the box alone)
  const int* zbox = nz == 512 ? box : nullptr;
  const int* ybox = ny == 512 ? box : nullptr;
  const float* khat = shell0 >= 0 ? p.khat + (size_t)shell0 * p.khat_stride : nullptr;
  if (shell0 >= 0 && p.spec_direct) {
    // read: the box's planes of the spectrum and the groups' tables;
    // written: the box's planes of every shell (or every plane)
    const double rowb = 8.0 * (double)ny * p.px;  // bytes of one plane of the spectrum
    const int g0 = shell0 / kZconvGroup, g1 = (shell0 + nshells + kZconvGroup - 1) / kZconvGroup;
    const double tables = 4.0 * (double)(g1 - g0) * (double)p.kz_group_stride;
    ProfScope ps(p, ST_Z_CONV, tables + (box ? 0.0 : (1.0 + nshells) * rowb * nz), 0.0, (1.0 + nshells) * rowb, box,
                 st);
    launch_zconv(p, spec, shell0, nshells, tmp, p.spec_elems, p.spec_in_box, box, st);
  } else {
    const double base = 8.0 * H + nshells * (khat ? 4.0 * (double)p.oct_elems : 0.0);
    // written: every plane, or the box's planes
    ProfScope ps(p, ST_FFT_Z_INV_MUL, base + (zbox ? 0.0 : nshells * 8.0 * H), 0.0, nshells * row * ny, zbox, st);
    StridedView v{(int64_t)ny * p.px, 0, ny * p.px, 1};
    KhatArgs K{khat, p.khat_stride, p.px, ny, nz, p.oct[1]};
    fft::launch_zmulti(nz, spec, tmp, p.spec_elems, nshells, v, p.fz, p.stw[2], p.twm, K, p.sm_count, st, zbox,
                       p.tune.zreg_cols);
  }
  {
    // read: the box's planes; written: their box rows (fused plans, whose
    // x pass visits the box's rows) or every row of them (the bank's planes
    // are summed whole)
    const bool rows_only = p.fused;
    ProfScope ps(p, ST_FFT_Y_INV, ybox ? 0.0 : nshells * 16.0 * H, rows_only ? nshells * row : 0.0,
                 (rows_only ? 1.0 : 2.0) * nshells * row * ny, ybox, st);
    StridedView v{p.px, (int64_t)ny * p.px, p.px, (int64_t)nz * nshells};
    fft::launch_strided(ny, true, tmp, tmp, v, p.fy, p.stw[1], p.tw[1], nshells > 1 ? p.tune.yinv_cols : p.tune.fwd_cols,
                        p.sm_count, st, ybox, nz,
                        fft::kPrunePlanes | (rows_only ? fft::kPruneOutY : 0));
  }
}

// The whole inverse: the z and y passes, then the x pass from tmp[s] into
// real fields out + s * out_stride.
void launch_fft_inverse(const Plan& p, const float2* spec, int shell0, int nshells, float2* tmp, float* out,
                        int64_t out_stride, cudaStream_t st, const int* box) {
  const int nx = p.grid.n[0], ny = p.grid.n[1], nz = p.grid.n[2];
  const double H = (double)nz * ny * (nx / 2 + 1);
  launch_inverse_zy(p, spec, shell0, nshells, tmp, st, box);
  {
    const int64_t rows = (int64_t)ny * nz * nshells;
    // every row, or the rows of the box's planes
    ProfScope ps(p, ST_FFT_X_C2R, box ? 0.0 : nshells * (4.0 * (double)p.nc + 8.0 * H), 0.0,
                 nshells * (double)ny * (4.0 * nx + 8.0 * (nx / 2 + 1)), box, st);
    fft::launch_x_c2r(nx / 2, tmp, out, nx, p.px, rows, (int64_t)ny * nz, out_stride, p.fx_half, p.stw[0],
                      p.tw[0], p.sm_count, st, box, ny);
  }
}

// ---------------------------------------------------------------------------
// Kernel spectra (Sec. 2.3): K_s depends only on |m|, so it is even in every
// axis and its DFT is the real separable cosine sum
//   K^_s(k) = sum_m K_s(m) cos(2 pi kx mx/nx) cos(2 pi ky my/ny) cos(2 pi kz mz/nz),
// evaluated over m >= 0 with weights 1 (m = 0) or 2 (m > 0) folded into the
// cosine tables, in FP64, in three passes (x, y, z), then divided by N_c.

__global__ void khat_pass_x(const double* __restrict__ Kc, const double* __restrict__ Cx, double* __restrict__ A1,
                            int ns, int H1, int ox) {
  const int64_t total = (int64_t)ns * H1 * H1 * ox;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(t % ox);
    const int64_t r = t / ox;  // (s, mz, my)
    const double* k = Kc + r * H1;
    const double* c = Cx + (int64_t)kx * H1;
    double acc = 0.0;
    for (int m = 0; m < H1; ++m) acc = fma(k[m], c[m], acc);
    A1[t] = acc;
  }
}

__global__ void khat_pass_y(const double* __restrict__ A1, const double* __restrict__ Cy, double* __restrict__ A2,
                            int ns, int H1, int oy, int ox) {
  const int64_t total = (int64_t)ns * H1 * oy * ox;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(t % ox);
    const int ky = (int)((t / ox) % oy);
    const int64_t smz = t / ((int64_t)ox * oy);  // (s, mz)
    const double* a = A1 + smz * H1 * ox + kx;
    const double* c = Cy + (int64_t)ky * H1;
    double acc = 0.0;
    for (int m = 0; m < H1; ++m) acc = fma(a[(int64_t)m * ox], c[m], acc);
    A2[t] = acc;
  }
}

// Writes the octant with rows padded to the pitch px (zeros for kx >= ox).
__global__ void khat_pass_z(const double* __restrict__ A2, const double* __restrict__ Cz, float* __restrict__ khat,
                            int ns, int H1, int oz, int oy, int ox, int px, double inv_nc) {
  const int64_t plane = (int64_t)oy * ox;
  const int64_t total = (int64_t)ns * oz * oy * px;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(t % px);
    const int64_t r = t / px;  // (s, kz, ky)
    const int ky = (int)(r % oy);
    const int kz = (int)((r / oy) % oz);
    const int s = (int)(r / ((int64_t)oy * oz));
    if (kx >= ox) {
      khat[t] = 0.0f;
      continue;
    }
    const double* a = A2 + (int64_t)s * H1 * plane + (int64_t)ky * ox + kx;
    const double* c = Cz + (int64_t)kz * H1;
    double acc = 0.0;
    for (int m = 0; m < H1; ++m) acc = fma(a[(int64_t)m * plane], c[m], acc);
    khat[t] = (float)(acc * inv_nc);
  }
}

// Host: cos(2 pi k m / n) with the argument reduced exactly (k m mod n).
static void cos_table(int n, int ok, int H1, std::vector<double>& out) {
  out.assign((size_t)ok * H1, 0.0);
  for (int k = 0; k < ok; ++k)
    for (int m = 0; m < H1; ++m) {
      const long long r = ((long long)k * m) % n;
      const double w = m == 0 ? 1.0 : 2.0;
      out[(size_t)k * H1 + m] = w * cos(2.0 * M_PI * (double)r / (double)n);
    }
}

ck_status build_kernel_spectra(Plan& p, cudaStream_t st) {
  const int H1 = p.H + 1;
  const int ns = p.ns;
  std::vector<double> Kc((size_t)ns * H1 * H1 * H1, 0.0);
  for (int s = 0; s < ns; ++s) {
    const std::vector<int>& o = p.offsets[s];
    for (size_t i = 0; i < o.size(); i += 3) {
      const int mx = o[i], my = o[i + 1], mz = o[i + 2];
      if (mx < 0 || my < 0 || mz < 0) continue;  // even in every axis: keep m >= 0
      Kc[(((size_t)s * H1 + mz) * H1 + my) * H1 + mx] = 1.0;
    }
  }
  std::vector<double> Cx, Cy, Cz;
  cos_table(p.grid.n[0], p.oct[0], H1, Cx);
  cos_table(p.grid.n[1], p.oct[1], H1, Cy);
  cos_table(p.grid.n[2], p.oct[2], H1, Cz);
  double* scratch = reinterpret_cast<double*>(p.bank);
  double* dK = scratch;
  double* dA1 = dK + Kc.size();
  double* dA2 = dA1 + (size_t)ns * H1 * H1 * p.oct[0];
  double* dCx = dA2 + (size_t)ns * H1 * p.oct[1] * p.oct[0];
  double* dCy = dCx + Cx.size();
  double* dCz = dCy + Cy.size();
  cudaError_t e = cudaMemcpyAsync(dK, Kc.data(), Kc.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dCx, Cx.data(), Cx.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dCy, Cy.data(), Cy.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dCz, Cz.data(), Cz.size() * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  const unsigned blocks = (unsigned)std::max(1, p.sm_count * 8);
  khat_pass_x<<<blocks, 256, 0, st>>>(dK, dCx, dA1, ns, H1, p.oct[0]);
  khat_pass_y<<<blocks, 256, 0, st>>>(dA1, dCy, dA2, ns, H1, p.oct[1], p.oct[0]);
  khat_pass_z<<<blocks, 256, 0, st>>>(dA2, dCz, p.khat, ns, H1, p.oct[2], p.oct[1], p.oct[0], p.px,
                                      1.0 / (double)p.nc);
  // the direct z step's table: the (x, y) sums per plane offset
  e = launch_zconv_table(p, dA2, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  // the host vectors must outlive the copies
  return cuda_status(cudaStreamSynchronize(st));
}

}  // namespace ck
