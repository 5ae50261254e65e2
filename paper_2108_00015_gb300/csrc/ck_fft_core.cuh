// ck_fft_core.cuh -- device code of the batched 3D FFT passes (Sec. 2.4:
// W_i = N *** K_i evaluated by FFT).  Included by the translation units that
// instantiate the passes for each transform length.
//
// Every pass transforms one axis.  A tile is kT = 8 independent lines of
// length L <= 512 held in shared memory (column layout s[l * kT + c] for the
// strided axes, row layout s[c * LP + l] for the x axis).  Persistent CTAs of
// 256 threads walk the tiles; the next tile is fetched with cp.async into a
// second buffer while the current one is transformed in place: in each
// mixed-radix (2, 3, 4, 5, 8) Stockham iteration every thread first reads its
// butterflies' inputs into registers, the block synchronises, and then the
// outputs are written in sorted order.  For the lengths the workloads use
// (template argument LC > 0) the radix schedule and all index arithmetic are
// compile-time constants; LC = 0 is the runtime fallback for any other
// length.  Strided axes (y, z) move rows of 8 contiguous complex values; the x
// axis reads contiguous real rows and runs a half-length complex transform
// with the even/odd split of a real sequence.
#pragma once

#include <math.h>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {
namespace fft {

constexpr int kThreads = 256;
constexpr int kT = 8;        // lines per tile

// Resident CTAs per SM the compile-time kernels are built for: 3 for lengths
// that are powers of two (<= 85 registers), 2 for those with radix 3 or 5.
__host__ __device__ constexpr int min_blocks(int L) { return L <= 0 ? 1 : ((L & (L - 1)) == 0 ? 3 : 2); }

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
  const float2 m2 = cscale(cmul_mi<INV>(t2), kSin60);  // -+ i sin(60) t2
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

// ---------------------------------------------------------------------------
// One Stockham iteration: radix R, Ns = product of the radices already
// applied, in place on kT lines of length L.  Twiddles tw[t * TWS] =
// e^{-2 pi i t / (L * TWS)}.  Element (l, c) of line c sits at
// s[l * kT + c] (column layout, strided passes; consecutive threads take
// consecutive lines) or s[c * LP + l] (row layout, x passes; consecutive
// threads take consecutive butterflies of one line).

__host__ __device__ constexpr int span_before(const RPlan& p, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= p.r[i];
  return ns;
}

template <bool ROW, int NBF>
__device__ __forceinline__ void split_b(int b, int nbf_rt, int& c, int& j) {
  const int nbf = NBF > 0 ? NBF : nbf_rt;
  if (ROW) { c = b / nbf; j = b - c * nbf; }
  else { c = b % kT; j = b / kT; }
}

template <bool ROW>
__device__ __forceinline__ int at(int l, int c, int lp) { return ROW ? c * lp + l : l * kT + c; }

template <int L, int S, bool INV, bool ROW, int LP, int TWS>
__device__ __forceinline__ void stage_ct(float2* s, const float2* tw) {
  constexpr RPlan P = rplan(L);
  constexpr int R = P.r[S];
  constexpr int Ns = span_before(P, S);
  constexpr int nbf = L / R;
  constexpr int total = nbf * kT;
  constexpr int NB = (total + kThreads - 1) / kThreads;
  constexpr int twstep = (L / (Ns * R)) * TWS;
  float2 v[NB][R];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (total % kThreads == 0 || b < total) {
      int c, j;
      split_b<ROW, nbf>(b, nbf, c, j);
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = s[at<ROW>(j + r * nbf, c, LP)];
      if constexpr (Ns > 1) {
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
  for (int q = 0; q < NB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (total % kThreads == 0 || b < total) {
      int c, j;
      split_b<ROW, nbf>(b, nbf, c, j);
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[at<ROW>(base + r * Ns, c, LP)] = v[q][r];
    }
  }
  __syncthreads();
}

template <int L, int S, bool INV, bool ROW, int LP, int TWS>
__device__ __forceinline__ void fft_ct(float2* s, const float2* tw) {
  constexpr RPlan P = rplan(L);
  if constexpr (S < P.nst) {
    if constexpr (P.r[S] != 1) stage_ct<L, S, INV, ROW, LP, TWS>(s, tw);
    fft_ct<L, S + 1, INV, ROW, LP, TWS>(s, tw);
  }
}

// Runtime-length fallback: the same iteration with runtime R, Ns, L.
template <int R, bool INV, bool ROW>
__device__ __forceinline__ void stage_rt(float2* s, const float2* tw, int tws, int L, int Ns, int lp) {
  constexpr int MAXB = (512 * kT / kThreads + R - 1) / R;
  const int nbf = L / R;
  const int total = nbf * kT;
  const int twstep = (L / (Ns * R)) * tws;
  float2 v[MAXB][R];
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (b < total) {
      int c, j;
      split_b<ROW, 0>(b, nbf, c, j);
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = s[at<ROW>(j + r * nbf, c, lp)];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[r * k * twstep];
        if (INV) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
      dft<R, INV>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (b < total) {
      int c, j;
      split_b<ROW, 0>(b, nbf, c, j);
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[at<ROW>(base + r * Ns, c, lp)] = v[q][r];
    }
  }
  __syncthreads();
}

template <bool INV, bool ROW>
__device__ __forceinline__ void fft_rt(float2* s, const float2* tw, int tws, const FftLen& f, int lp) {
  int Ns = 1;
  for (int i = 0; i < f.nst; ++i) {
    switch (f.radix[i]) {
      case 2: stage_rt<2, INV, ROW>(s, tw, tws, f.n, Ns, lp); break;
      case 3: stage_rt<3, INV, ROW>(s, tw, tws, f.n, Ns, lp); break;
      case 4: stage_rt<4, INV, ROW>(s, tw, tws, f.n, Ns, lp); break;
      case 5: stage_rt<5, INV, ROW>(s, tw, tws, f.n, Ns, lp); break;
      case 8: stage_rt<8, INV, ROW>(s, tw, tws, f.n, Ns, lp); break;
      default: break;  // radix 1: identity
    }
    Ns *= f.radix[i];
  }
}

// Column-layout transform of kT lines (strided passes).
template <int LC, bool INV>
__device__ __forceinline__ void fft_cols(float2* s, const float2* tw, const FftLen& f) {
  if constexpr (LC > 0) fft_ct<LC, 0, INV, false, 0, 1>(s, tw);
  else fft_rt<INV, false>(s, tw, 1, f, 0);
}

// Row pitch of the x-pass tiles: M + 2 complex (even: 16-byte aligned rows).
__host__ __device__ constexpr int row_pitch(int M) { return M + 2; }

// Row-layout transform of kT lines of length M (x passes; twiddles of 2M).
template <int MC, bool INV>
__device__ __forceinline__ void fft_rows(float2* s, const float2* tw, const FftLen& f) {
  if constexpr (MC > 0) fft_ct<MC, 0, INV, true, row_pitch(MC), 2>(s, tw);
  else fft_rt<INV, true>(s, tw, 2, f, row_pitch(f.n));
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // 0 source bytes: the destination is zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Kernel spectra for the fused multiply: the octant K^_s[kzf][kyf][kx] with
// rows padded to the spectrum pitch px (zeros for kx > n[0]/2).  Element
// (kz, i) of the z pass, i = ky * px + kx, uses (min(kz, nz-kz),
// min(ky, ny-ky), kx).
struct KhatArgs {
  const float* khat;  // octant of shell 0 (nullptr: multiply by 1)
  int64_t shell_stride;
  int px, ny, nz, oy;
};

// A strided-axis view: element (o, l, i) at o*so + l*sl + i, l in [0, L),
// i in [0, inner); a tile is one o and kT consecutive i.
struct StridedView {
  int64_t sl, so;
  int inner;
  int64_t n_outer;
};

__device__ __forceinline__ void load_strided_tile(float2* s, const float2* in, const StridedView& v, int L,
                                                  int64_t tile) {
  const int tpo = (v.inner + kT - 1) / kT;
  const int64_t o = tile / tpo;
  const int i0 = (int)(tile - o * tpo) * kT;
  const float2* base = in + o * v.so + i0;
  for (int idx = threadIdx.x; idx < L * (kT / 2); idx += kThreads) {
    const int l = idx / (kT / 2), c = (idx % (kT / 2)) * 2;
    const bool ok = i0 + c < v.inner;
    cp_async16(s + l * kT + c, ok ? base + (int64_t)l * v.sl + c : in, ok);
  }
}

__device__ __forceinline__ void store_strided_tile(const float2* s, float2* out, const StridedView& v, int L,
                                                   int64_t tile) {
  const int tpo = (v.inner + kT - 1) / kT;
  const int64_t o = tile / tpo;
  const int i0 = (int)(tile - o * tpo) * kT;
  float2* base = out + o * v.so + i0;
  for (int idx = threadIdx.x; idx < L * (kT / 2); idx += kThreads) {
    const int l = idx / (kT / 2), c = (idx % (kT / 2)) * 2;
    if (i0 + c < v.inner) {
      const float2 a = s[l * kT + c], b = s[l * kT + c + 1];
      *reinterpret_cast<float4*>(base + (int64_t)l * v.sl + c) = make_float4(a.x, a.y, b.x, b.y);
    }
  }
}

// ---------------------------------------------------------------------------
// kernels

// Strided-axis transform (in place allowed), persistent with a prefetched
// second tile buffer.
template <int LC, bool INV>
__global__ void __launch_bounds__(kThreads, min_blocks(LC))
    strided_kernel(const float2* in, float2* out, StridedView v, FftLen f, const float2* __restrict__ tw) {
  extern __shared__ float4 smem4[];
  const int L = LC > 0 ? LC : f.n;
  float2* buf0 = reinterpret_cast<float2*>(smem4);
  float2* buf1 = buf0 + L * kT;
  float2* tws = buf1 + L * kT;
  const int64_t ntiles = v.n_outer * ((v.inner + kT - 1) / kT);
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  for (int i = threadIdx.x; i < L; i += kThreads) tws[i] = __ldg(tw + i);
  load_strided_tile(buf0, in, v, L, t);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it) {
    const int64_t tn = t + gridDim.x;
    float2* cur = (it & 1) ? buf1 : buf0;
    if (tn < ntiles) load_strided_tile((it & 1) ? buf0 : buf1, in, v, L, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    fft_cols<LC, INV>(cur, tws, f);
    store_strided_tile(cur, out, v, L, t);
    __syncthreads();
    t = tn;
  }
}

// Inverse z pass of every shell at once: a half-spectrum tile is read once,
// then for each shell s it is multiplied by K^_s (Eq. 9 in Fourier space),
// transformed along z and stored to that shell's scratch spectrum
// out + s * out_stride.  The tile's slab of K^_s (nz/2 + 1 rows of kT
// values) is fetched with cp.async while the previous shell is transformed.
// khat == nullptr: one transform, factor 1.
template <int LC>
__global__ void __launch_bounds__(kThreads, min_blocks(LC))
    zmulti_kernel(const float2* in, float2* out, int64_t out_stride, int nshells, StridedView v, FftLen f,
                  const float2* __restrict__ tw, KhatArgs K) {
  extern __shared__ float4 smem4[];
  const int L = LC > 0 ? LC : f.n;
  const int OZ = L / 2 + 1;
  float2* pristine = reinterpret_cast<float2*>(smem4);
  float2* work = pristine + L * kT;
  float2* tws = work + L * kT;
  float* slab0 = reinterpret_cast<float*>(tws + L);
  float* slab1 = slab0 + OZ * kT;
  const int64_t ntiles = (v.inner + kT - 1) / kT;
  for (int i = threadIdx.x; i < L; i += kThreads) tws[i] = __ldg(tw + i);
  // two halves of 4 columns per tile: px is a multiple of 4 and i0 of 8, so
  // each half lies in one ky row of the spectrum
  auto load_slab = [&](float* dst, int s, int64_t tile) {
    const float* kh = K.khat + (int64_t)s * K.shell_stride;
    for (int idx = threadIdx.x; idx < 2 * OZ; idx += kThreads) {
      const int kzf = idx >> 1, h = idx & 1;
      const int i = (int)tile * kT + 4 * h;
      const bool ok = i < v.inner;
      const int ky = i / K.px, kx = i - (i / K.px) * K.px;
      const int kyf = min(ky, K.ny - ky);
      cp_async16(dst + kzf * kT + 4 * h, ok ? kh + ((int64_t)kzf * K.oy + kyf) * K.px + kx : K.khat, ok);
    }
  };
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    load_strided_tile(pristine, in, v, L, t);
    if (K.khat) load_slab(slab0, 0, t);
    cp_async_commit();
    for (int s = 0; s < nshells; ++s) {
      const float* slab = (s & 1) ? slab1 : slab0;
      if (K.khat && s + 1 < nshells) load_slab((s & 1) ? slab0 : slab1, s + 1, t);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      for (int idx = threadIdx.x; idx < L * kT; idx += kThreads) {
        const int l = idx / kT, c = idx % kT;
        const float m = K.khat ? slab[min(l, L - l) * kT + c] : 1.0f;
        work[idx] = cscale(pristine[idx], m);
      }
      __syncthreads();
      fft_cols<LC, true>(work, tws, f);
      store_strided_tile(work, out + (int64_t)s * out_stride, v, L, t);
      __syncthreads();
    }
  }
}

// Forward x pass: real rows of length nx = 2M -> half-spectrum rows (pitch
// px).  z[m] = x[2m] + i x[2m+1], Z = DFT_M(z), then X[k] = E[k] +
// e^{-2 pi i k/nx} O[k], E = (Z[k] + conj Z[M-k]) / 2,
// O = (Z[k] - conj Z[M-k]) / 2i, k = 0..M.  Tiles of kT rows in row layout.
template <int MC>
__global__ void __launch_bounds__(kThreads, min_blocks(MC))
    x_r2c_kernel(const float* __restrict__ in, float2* __restrict__ out, int nx, int px, int64_t rows, FftLen f,
                 const float2* __restrict__ tw) {
  extern __shared__ float4 smem4[];
  const int M = MC > 0 ? MC : nx / 2;
  const int NX = 2 * M;
  const int LP = row_pitch(M);
  float2* buf0 = reinterpret_cast<float2*>(smem4);
  float2* buf1 = buf0 + kT * LP;
  float2* tws = buf1 + kT * LP;
  const int64_t ntiles = (rows + kT - 1) / kT;
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  for (int i = threadIdx.x; i < NX; i += kThreads) tws[i] = __ldg(tw + i);
  auto load = [&](float2* s, int64_t tile) {
    const int64_t r0 = tile * kT;
    if (M % 2 == 0) {  // rows 16-byte aligned: two z values per copy
      const int np = M / 2;
      for (int idx = threadIdx.x; idx < kT * np; idx += kThreads) {
        const int c = idx / np, m = 2 * (idx - c * np);
        const bool ok = r0 + c < rows;
        cp_async16(s + c * LP + m, ok ? (const void*)(in + (r0 + c) * NX + 2 * m) : (const void*)in, ok);
      }
    } else {
      for (int idx = threadIdx.x; idx < kT * M; idx += kThreads) {
        const int c = idx / M, m = idx - c * M;
        const bool ok = r0 + c < rows;
        cp_async8(s + c * LP + m, ok ? (const void*)(in + (r0 + c) * NX + 2 * m) : (const void*)in, ok);
      }
    }
  };
  load(buf0, t);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it) {
    const int64_t tn = t + gridDim.x;
    float2* s = (it & 1) ? buf1 : buf0;
    if (tn < ntiles) load((it & 1) ? buf0 : buf1, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    fft_rows<MC, false>(s, tws, f);
    const int64_t r0 = t * kT;
    for (int idx = threadIdx.x; idx < kT * px; idx += kThreads) {
      const int c = idx / px, k = idx - c * px;
      const int64_t row = r0 + c;
      if (row >= rows) continue;
      float2 X = make_float2(0.f, 0.f);
      if (k <= M) {
        const float2 zk = s[c * LP + (k == M ? 0 : k)];
        const float2 zc = cconj(s[c * LP + (k == 0 ? 0 : M - k)]);
        const float2 E = cscale(cadd(zk, zc), 0.5f);
        const float2 O = cscale(cmul_mi<false>(csub(zk, zc)), 0.5f);
        X = cadd(E, cmul(tws[k], O));
      }
      out[row * px + k] = X;
    }
    __syncthreads();
    t = tn;
  }
}

// Inverse x pass: half-spectrum rows -> real rows.  With w^-k =
// e^{+2 pi i k/nx}: Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k]),
// z = IDFT_M(Z) (unnormalised), x[2m] = Re z[m], x[2m+1] = Im z[m].  Input
// rows are contiguous (pitch px); output row r goes to
// out + (r / rows_per_shell) * out_shell_stride + (r % rows_per_shell) * nx.
template <int MC>
__global__ void __launch_bounds__(kThreads, min_blocks(MC))
    x_c2r_kernel(const float2* __restrict__ in, float* __restrict__ out, int nx, int px, int64_t rows,
                 int64_t rows_per_shell, int64_t out_shell_stride, FftLen f, const float2* __restrict__ tw) {
  extern __shared__ float4 smem4[];
  const int M = MC > 0 ? MC : nx / 2;
  const int NX = 2 * M;
  const int LP = row_pitch(M);
  float2* buf0 = reinterpret_cast<float2*>(smem4);
  float2* buf1 = buf0 + kT * LP;
  float2* tws = buf1 + kT * LP;
  const int64_t ntiles = (rows + kT - 1) / kT;
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  for (int i = threadIdx.x; i < NX; i += kThreads) tws[i] = __ldg(tw + i);
  // X[0..M] as pairs (k, k+1), k even: M/2 + 1 copies per row; for even M
  // the last pair also reads padding column M + 1 (< px)
  const int np = M / 2 + 1;
  auto load = [&](float2* s, int64_t tile) {
    const int64_t r0 = tile * kT;
    for (int idx = threadIdx.x; idx < kT * np; idx += kThreads) {
      const int c = idx / np, k = 2 * (idx - c * np);
      const bool ok = r0 + c < rows;
      cp_async16(s + c * LP + k, ok ? (const void*)(in + (r0 + c) * px + k) : (const void*)in, ok);
    }
  };
  load(buf0, t);
  cp_async_commit();
  const int half = M / 2 + 1;
  for (int it = 0; t < ntiles; ++it) {
    const int64_t tn = t + gridDim.x;
    float2* s = (it & 1) ? buf1 : buf0;
    if (tn < ntiles) load((it & 1) ? buf0 : buf1, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    for (int idx = threadIdx.x; idx < kT * half; idx += kThreads) {
      const int c = idx / half, k = idx - c * half;
      const float2 a = s[c * LP + k];
      const float2 b = s[c * LP + M - k];
      const float2 ca = cconj(a), cb = cconj(b);
      const float2 zk = cadd(cadd(a, cb), cmul_mi<true>(cmul(cconj(tws[k]), csub(a, cb))));
      s[c * LP + k] = zk;
      if (k != 0 && 2 * k != M) {
        const float2 zm = cadd(cadd(b, ca), cmul_mi<true>(cmul(cconj(tws[M - k]), csub(b, ca))));
        s[c * LP + M - k] = zm;
      }
    }
    __syncthreads();
    fft_rows<MC, true>(s, tws, f);
    const int64_t r0 = t * kT;
    if (M % 2 == 0) {  // two z values (four reals) per 16-byte store
      const int nq = M / 2;
      for (int idx = threadIdx.x; idx < kT * nq; idx += kThreads) {
        const int c = idx / nq, m = 2 * (idx - c * nq);
        const int64_t row = r0 + c;
        if (row < rows) {
          const int64_t sh = row / rows_per_shell, rr = row - sh * rows_per_shell;
          const float2 a = s[c * LP + m], b = s[c * LP + m + 1];
          *reinterpret_cast<float4*>(out + sh * out_shell_stride + rr * NX + 2 * m) = make_float4(a.x, a.y, b.x, b.y);
        }
      }
    } else {
      for (int idx = threadIdx.x; idx < kT * M; idx += kThreads) {
        const int c = idx / M, m = idx - c * M;
        const int64_t row = r0 + c;
        if (row < rows) {
          const int64_t sh = row / rows_per_shell, rr = row - sh * rows_per_shell;
          *reinterpret_cast<float2*>(out + sh * out_shell_stride + rr * NX + 2 * m) = s[c * LP + m];
        }
      }
    }
    __syncthreads();
    t = tn;
  }
}

// shared-memory bytes of each kernel
inline size_t strided_smem(int L) { return (size_t)L * (2 * kT + 1) * sizeof(float2); }
inline size_t zmulti_smem(int L) {
  return (size_t)L * (2 * kT + 1) * sizeof(float2) + (size_t)2 * (L / 2 + 1) * kT * sizeof(float);
}
inline size_t xpass_smem(int nx) { return ((size_t)2 * kT * row_pitch(nx / 2) + nx) * sizeof(float2); }

// Launch helpers (one translation unit each; they pick the compile-time
// length when LC/MC is one of the instantiated lengths).
void launch_strided(int L, bool inv, const float2* in, float2* out, const StridedView& v, const FftLen& f,
                    const float2* tw, int sm_count, cudaStream_t st);
void launch_zmulti(int L, const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                   const FftLen& f, const float2* tw, const KhatArgs& K, int sm_count, cudaStream_t st);
void launch_x_r2c(int M, const float* in, float2* out, int nx, int px, int64_t rows, const FftLen& f,
                  const float2* tw, int sm_count, cudaStream_t st);
void launch_x_c2r(int M, const float2* in, float* out, int nx, int px, int64_t rows, int64_t rows_per_shell,
                  int64_t out_shell_stride, const FftLen& f, const float2* tw, int sm_count, cudaStream_t st);

// Persistent grid: the resident CTAs of every SM, at most one CTA per tile.
template <typename K>
inline unsigned persistent_grid(K kernel, size_t smem, int sm_count, int64_t ntiles) {
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int64_t g = std::min<int64_t>(ntiles, (int64_t)sm_count * occ);
  return (unsigned)std::max<int64_t>(g, 1);
}

template <typename K>
inline void allow_smem(K kernel, size_t smem) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace fft
}  // namespace ck
