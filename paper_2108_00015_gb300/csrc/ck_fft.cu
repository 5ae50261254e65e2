// ck_fft.cu -- the convolution stage (Sec. 2.4, Eqs. 9-10) by FFT: an
// in-house batched 3D real-to-complex / complex-to-real transform, the
// kernel-spectrum multiply fused into the first inverse pass, and the
// once-per-plan build of the shell spectra K^_s.
//
// Each pass transforms one axis.  A CTA loads a tile of 16 independent
// lines (length L <= 512) into shared memory, runs the mixed-radix (2, 3, 4,
// 5, 8) Stockham iterations there -- every butterfly reads its inputs from
// shared memory into registers, the block synchronises, then writes its
// outputs in sorted order -- and stores the tile back.  Strided axes (y, z)
// move rows of 16 contiguous complex values (128 bytes); the x axis reads
// contiguous real rows and uses a half-length complex transform with the
// even/odd split of a real sequence.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {

// ---------------------------------------------------------------------------
// small DFTs, exponent sign -1 (forward) or +1 (INV)

constexpr float kSqrtHalf = 0.70710678118654752440f;
constexpr float kSin60 = 0.86602540378443864676f;
constexpr float kC1_5 = 0.30901699437494742410f;   // cos(2 pi / 5)
constexpr float kC2_5 = -0.80901699437494742410f;  // cos(4 pi / 5)
constexpr float kS1_5 = 0.95105651629515357212f;   // sin(2 pi / 5)
constexpr float kS2_5 = 0.58778525229247312917f;   // sin(4 pi / 5)

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
  const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  const float2 t2 = cadd(v[1], v[3]), t3 = cmul_mi<INV>(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // o[k] *= w8^k, w8 = e^{-+ i pi / 4}
  const float s = INV ? kSqrtHalf : -kSqrtHalf;
  o[1] = make_float2(kSqrtHalf * o[1].x - s * o[1].y, s * o[1].x + kSqrtHalf * o[1].y);
  o[2] = cmul_mi<INV>(o[2]);
  o[3] = make_float2(-kSqrtHalf * o[3].x - s * o[3].y, -kSqrtHalf * o[3].y + s * o[3].x);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  const float2 t1 = cadd(v[1], v[2]);
  const float2 t2 = csub(v[1], v[2]);
  const float2 m1 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  // -+ i sin(60) t2
  const float2 m2 = cscale(cmul_mi<INV>(t2), kSin60);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m1, m2);
  v[2] = csub(m1, m2);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
  const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const float2 m1 = make_float2(v[0].x + kC1_5 * t1.x + kC2_5 * t2.x, v[0].y + kC1_5 * t1.y + kC2_5 * t2.y);
  const float2 m2 = make_float2(v[0].x + kC2_5 * t1.x + kC1_5 * t2.x, v[0].y + kC2_5 * t1.y + kC1_5 * t2.y);
  const float2 u1 = make_float2(kS1_5 * t3.x + kS2_5 * t4.x, kS1_5 * t3.y + kS2_5 * t4.y);
  const float2 u2 = make_float2(kS2_5 * t3.x - kS1_5 * t4.x, kS2_5 * t3.y - kS1_5 * t4.y);
  const float2 j1 = cmul_mi<INV>(u1), j2 = cmul_mi<INV>(u2);
  v[0] = make_float2(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
  v[1] = cadd(m1, j1);
  v[4] = csub(m1, j1);
  v[2] = cadd(m2, j2);
  v[3] = csub(m2, j2);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 5) dft5<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
}

constexpr int kThreads = 512;
constexpr int kT = 16;  // lines per tile

// One Stockham iteration of radix R on T lines of length L held in shared
// memory as s[l * TP + c].  Ns = product of the radices already applied.
// Twiddles come from tw[t * tws] = e^{-2 pi i t / L}.
template <int R, bool INV, int TP>
__device__ __forceinline__ void fft_stage(float2* s, const float2* tw, int tws, int L, int Ns) {
  constexpr int MAXB = (16 + R - 1) / R;  // L * kT / (R * kThreads) <= 16 / R for L <= 512
  const int nbf = L / R;
  const int total = nbf * kT;
  const int twstep = (L / (Ns * R)) * tws;
  float2 v[MAXB][R];
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (b < total) {
      const int c = b % kT, j = b / kT;
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = s[(j + r * nbf) * TP + c];
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * k * twstep];
          if (INV) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft<R, INV>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (b < total) {
      const int c = b % kT, j = b / kT;
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[(base + r * Ns) * TP + c] = v[q][r];
    }
  }
  __syncthreads();
}

template <bool INV, int TP>
__device__ __forceinline__ void fft_lines(float2* s, const float2* tw, int tws, const FftLen& f) {
  int Ns = 1;
  for (int i = 0; i < f.nst; ++i) {
    switch (f.radix[i]) {
      case 2: fft_stage<2, INV, TP>(s, tw, tws, f.n, Ns); break;
      case 3: fft_stage<3, INV, TP>(s, tw, tws, f.n, Ns); break;
      case 4: fft_stage<4, INV, TP>(s, tw, tws, f.n, Ns); break;
      case 5: fft_stage<5, INV, TP>(s, tw, tws, f.n, Ns); break;
      case 8: fft_stage<8, INV, TP>(s, tw, tws, f.n, Ns); break;
      default: break;  // radix 1: identity
    }
    Ns *= f.radix[i];
  }
}

// Kernel-spectrum lookup for the fused multiply: element (kz, i) of the
// z pass, i = ky * px + kx, reads the octant at (min(kz, nz-kz),
// min(ky, ny-ky), kx); kx beyond n[0]/2 (row padding) gets 0.
struct KhatArgs {
  const float* khat;
  int px, ny, nz, ox, oy;
};

__device__ __forceinline__ float khat_at(const KhatArgs& K, int kz, int i) {
  const int ky = i / K.px;
  const int kx = i - ky * K.px;
  if (kx >= K.ox) return 0.0f;
  const int kzf = min(kz, K.nz - kz);
  const int kyf = min(ky, K.ny - ky);
  return __ldg(K.khat + ((int64_t)kzf * K.oy + kyf) * K.ox + kx);
}

// Transform along a strided axis: element (o, l, i) at o*so + l*sl + i,
// l in [0, L), i in [0, inner).  One CTA = one outer index and 16
// consecutive inner indices.
template <bool INV, bool MUL>
__global__ void __launch_bounds__(kThreads, 1) fft_strided_kernel(const float2* in, float2* out, int64_t sl,
                                                               int64_t so, int inner, FftLen f,
                                                               const float2* __restrict__ tw, KhatArgs K) {
  extern __shared__ float4 smem4[];
  float2* s = reinterpret_cast<float2*>(smem4);
  float2* tws = s + f.n * kT;
  const int L = f.n;
  const int i0 = blockIdx.x * kT;
  const int64_t base = (int64_t)blockIdx.y * so + i0;
  for (int t = threadIdx.x; t < L; t += kThreads) tws[t] = __ldg(tw + t);
  for (int idx = threadIdx.x; idx < L * (kT / 2); idx += kThreads) {
    const int l = idx / (kT / 2), c = (idx % (kT / 2)) * 2;
    const int i = i0 + c;
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    const float2* src = in + base + (int64_t)l * sl + c;
    if (i + 1 < inner) {
      const float4 v = *reinterpret_cast<const float4*>(src);
      a = make_float2(v.x, v.y);
      b = make_float2(v.z, v.w);
    } else if (i < inner) {
      a = *src;
    }
    if (MUL) {
      if (i < inner) a = cscale(a, khat_at(K, l, i));
      if (i + 1 < inner) b = cscale(b, khat_at(K, l, i + 1));
    }
    s[l * kT + c] = a;
    s[l * kT + c + 1] = b;
  }
  __syncthreads();
  fft_lines<INV, kT>(s, tws, 1, f);
  for (int idx = threadIdx.x; idx < L * (kT / 2); idx += kThreads) {
    const int l = idx / (kT / 2), c = (idx % (kT / 2)) * 2;
    const int i = i0 + c;
    float2* dst = out + base + (int64_t)l * sl + c;
    const float2 a = s[l * kT + c], b = s[l * kT + c + 1];
    if (i + 1 < inner) {
      *reinterpret_cast<float4*>(dst) = make_float4(a.x, a.y, b.x, b.y);
    } else if (i < inner) {
      *dst = a;
    }
  }
}

constexpr int kTPx = kT + 1;  // padded line stride for the x pass

// Forward x pass: real rows of length nx -> half-spectrum rows (pitch px).
// z[m] = x[2m] + i x[2m+1], Z = DFT_M(z) (M = nx/2), then
// X[k] = E[k] + e^{-2 pi i k/nx} O[k] with E = (Z[k] + conj Z[M-k]) / 2 and
// O = (Z[k] - conj Z[M-k]) / 2i, for k = 0..M.
__global__ void __launch_bounds__(kThreads, 1) fft_x_r2c_kernel(const float* __restrict__ in, float2* __restrict__ out,
                                                             int nx, int px, int64_t rows, FftLen f,
                                                             const float2* __restrict__ tw) {
  extern __shared__ float4 smem4[];
  float2* s = reinterpret_cast<float2*>(smem4);
  const int M = nx / 2;
  float2* tws = s + (M + 1) * kTPx;
  const int64_t r0 = (int64_t)blockIdx.x * kT;
  for (int t = threadIdx.x; t < nx; t += kThreads) tws[t] = __ldg(tw + t);
  for (int idx = threadIdx.x; idx < kT * M; idx += kThreads) {
    const int c = idx / M, m = idx - c * M;
    const int64_t row = r0 + c;
    float2 z = make_float2(0.f, 0.f);
    if (row < rows) z = *reinterpret_cast<const float2*>(in + row * nx + 2 * m);
    s[m * kTPx + c] = z;
  }
  __syncthreads();
  fft_lines<false, kTPx>(s, tws, 2, f);
  for (int idx = threadIdx.x; idx < kT * px; idx += kThreads) {
    const int c = idx / px, k = idx - c * px;
    const int64_t row = r0 + c;
    if (row >= rows) continue;
    float2 X = make_float2(0.f, 0.f);
    if (k <= M) {
      const float2 zk = s[(k == M ? 0 : k) * kTPx + c];
      const float2 zc = cconj(s[(k == 0 ? 0 : M - k) * kTPx + c]);
      const float2 E = cscale(cadd(zk, zc), 0.5f);
      const float2 O = cscale(cmul_mi<false>(csub(zk, zc)), 0.5f);
      X = cadd(E, cmul(tws[k], O));
    }
    out[row * px + k] = X;
  }
}

// Inverse x pass: half-spectrum rows -> real rows.  With w^-k =
// e^{+2 pi i k/nx}: Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k]),
// z = IDFT_M(Z) (unnormalised), x[2m] = Re z[m], x[2m+1] = Im z[m].
__global__ void __launch_bounds__(kThreads, 1) fft_x_c2r_kernel(const float2* __restrict__ in, float* __restrict__ out,
                                                             int nx, int px, int64_t rows, FftLen f,
                                                             const float2* __restrict__ tw) {
  extern __shared__ float4 smem4[];
  float2* s = reinterpret_cast<float2*>(smem4);
  const int M = nx / 2;
  float2* tws = s + (M + 1) * kTPx;
  const int64_t r0 = (int64_t)blockIdx.x * kT;
  for (int t = threadIdx.x; t < nx; t += kThreads) tws[t] = __ldg(tw + t);
  for (int idx = threadIdx.x; idx < kT * (M + 1); idx += kThreads) {
    const int c = idx / (M + 1), k = idx - c * (M + 1);
    const int64_t row = r0 + c;
    s[k * kTPx + c] = row < rows ? in[row * px + k] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int half = M / 2 + 1;
  for (int idx = threadIdx.x; idx < kT * half; idx += kThreads) {
    const int c = idx / half, k = idx - c * half;
    const float2 a = s[k * kTPx + c];
    const float2 b = s[(M - k) * kTPx + c];
    const float2 ca = cconj(a), cb = cconj(b);
    const float2 zk = cadd(cadd(a, cb), cmul_mi<true>(cmul(cconj(tws[k]), csub(a, cb))));
    s[k * kTPx + c] = zk;
    if (k != 0 && 2 * k != M) {
      const float2 zm = cadd(cadd(b, ca), cmul_mi<true>(cmul(cconj(tws[M - k]), csub(b, ca))));
      s[(M - k) * kTPx + c] = zm;
    }
  }
  __syncthreads();
  fft_lines<true, kTPx>(s, tws, 2, f);
  for (int idx = threadIdx.x; idx < kT * M; idx += kThreads) {
    const int c = idx / M, m = idx - c * M;
    const int64_t row = r0 + c;
    if (row < rows) *reinterpret_cast<float2*>(out + row * nx + 2 * m) = s[m * kTPx + c];
  }
}

static size_t strided_smem(int L) { return (size_t)L * (kT + 1) * sizeof(float2); }
static size_t xpass_smem(int nx) { return ((size_t)(nx / 2 + 1) * kTPx + nx) * sizeof(float2); }

ck_status fft_init_attributes() {
  const int maxs = (int)strided_smem(512);
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(fft_strided_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_strided_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fft_strided_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
  return cuda_status(e);
}

static void strided(const Plan& p, bool inv, bool mul, const float2* in, float2* out, int axis,
                    const float* khat, cudaStream_t st) {
  const int nx = p.grid.n[0], ny = p.grid.n[1], nz = p.grid.n[2];
  const double H = (double)nz * ny * (nx / 2 + 1);  // useful complex values
  const int stage = axis == 1 ? (inv ? ST_FFT_Y_INV : ST_FFT_Y_FWD) : (inv ? ST_FFT_Z_INV_MUL : ST_FFT_Z_FWD);
  ProfScope ps(p, stage, 16.0 * H + (mul ? 4.0 * (double)p.oct_elems : 0.0), st);
  KhatArgs K{khat, p.px, ny, nz, p.oct[0], p.oct[1]};
  if (axis == 1) {
    dim3 grid((unsigned)((p.px + kT - 1) / kT), (unsigned)nz);
    const size_t sm = strided_smem(ny);
    if (inv)
      fft_strided_kernel<true, false><<<grid, kThreads, sm, st>>>(in, out, p.px, (int64_t)ny * p.px, p.px,
                                                                  p.fy, p.tw[1], K);
    else
      fft_strided_kernel<false, false><<<grid, kThreads, sm, st>>>(in, out, p.px, (int64_t)ny * p.px, p.px,
                                                                   p.fy, p.tw[1], K);
  } else {
    const int inner = ny * p.px;
    dim3 grid((unsigned)((inner + kT - 1) / kT), 1);
    const size_t sm = strided_smem(nz);
    if (inv && mul)
      fft_strided_kernel<true, true><<<grid, kThreads, sm, st>>>(in, out, inner, 0, inner, p.fz, p.tw[2], K);
    else if (inv)
      fft_strided_kernel<true, false><<<grid, kThreads, sm, st>>>(in, out, inner, 0, inner, p.fz, p.tw[2], K);
    else
      fft_strided_kernel<false, false><<<grid, kThreads, sm, st>>>(in, out, inner, 0, inner, p.fz, p.tw[2], K);
  }
}

void launch_fft_forward(const Plan& p, const float* in, float2* spec, cudaStream_t st) {
  const int nx = p.grid.n[0];
  const int64_t rows = (int64_t)p.grid.n[1] * p.grid.n[2];
  {
  ProfScope ps(p, ST_FFT_X_R2C, 4.0 * (double)p.nc + 8.0 * (double)rows * (nx / 2 + 1), st);
  fft_x_r2c_kernel<<<(unsigned)((rows + kT - 1) / kT), kThreads, xpass_smem(nx), st>>>(in, spec, nx, p.px, rows,
                                                                                       p.fx_half, p.tw[0]);
  }
  strided(p, false, false, spec, spec, 1, nullptr, st);
  strided(p, false, false, spec, spec, 2, nullptr, st);
}

void launch_fft_inverse(const Plan& p, const float2* spec, const float* khat_shell, float2* tmp, float* out,
                        cudaStream_t st) {
  const int nx = p.grid.n[0];
  const int64_t rows = (int64_t)p.grid.n[1] * p.grid.n[2];
  strided(p, true, khat_shell != nullptr, spec, tmp, 2, khat_shell, st);
  strided(p, true, false, tmp, tmp, 1, nullptr, st);
  ProfScope ps(p, ST_FFT_X_C2R, 4.0 * (double)p.nc + 8.0 * (double)rows * (nx / 2 + 1), st);
  fft_x_c2r_kernel<<<(unsigned)((rows + kT - 1) / kT), kThreads, xpass_smem(nx), st>>>(tmp, out, nx, p.px, rows,
                                                                                       p.fx_half, p.tw[0]);
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

__global__ void khat_pass_z(const double* __restrict__ A2, const double* __restrict__ Cz, float* __restrict__ khat,
                            int ns, int H1, int oz, int oy, int ox, double inv_nc) {
  const int64_t plane = (int64_t)oy * ox;
  const int64_t total = (int64_t)ns * oz * plane;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t yx = t % plane;
    const int kz = (int)((t / plane) % oz);
    const int s = (int)(t / (plane * oz));
    const double* a = A2 + (int64_t)s * H1 * plane + yx;
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
  khat_pass_z<<<blocks, 256, 0, st>>>(dA2, dCz, p.khat, ns, H1, p.oct[2], p.oct[1], p.oct[0], 1.0 / (double)p.nc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  // the host vectors must outlive the copies
  return cuda_status(cudaStreamSynchronize(st));
}

}  // namespace ck
