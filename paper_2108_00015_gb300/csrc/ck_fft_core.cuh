// ck_fft_core.cuh -- device code of the batched 3D FFT passes (Sec. 2.4:
// W_i = N *** K_i evaluated by FFT).  Included by the translation units that
// instantiate the passes for each transform length.
//
// Every pass transforms one axis.  A tile is kT = 8 independent lines of
// length L <= 512 held in shared memory in the column layout s[l * kT + c].  Persistent CTAs of
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

// x * e^{-+ i theta} (forward: c - i s, INV: c + i s), (c, s) = (cos theta, sin theta)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 x, float c, float s) {
  return INV ? make_float2(x.x * c - x.y * s, x.x * s + x.y * c) : make_float2(x.x * c + x.y * s, x.y * c - x.x * s);
}

constexpr float kC1_16 = 0.92387953251128675613f;  // cos(pi / 8)
constexpr float kS1_16 = 0.38268343236508977173f;  // sin(pi / 8)

// 16 points as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2; DFT over n1, twiddle
// w16^(n2 k1), DFT over n2.  Natural order in and out.
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  float2 a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[4 * n1 + n2];
    dft4<INV>(a[n2]);
  }
  a[1][1] = rot<INV>(a[1][1], kC1_16, kS1_16);        // w^1
  a[1][2] = rot<INV>(a[1][2], kSqrtHalf, kSqrtHalf);  // w^2
  a[1][3] = rot<INV>(a[1][3], kS1_16, kC1_16);        // w^3
  a[2][1] = rot<INV>(a[2][1], kSqrtHalf, kSqrtHalf);  // w^2
  a[2][2] = cmul_mi<INV>(a[2][2]);                    // w^4
  a[2][3] = rot<INV>(a[2][3], -kSqrtHalf, kSqrtHalf); // w^6
  a[3][1] = rot<INV>(a[3][1], kS1_16, kC1_16);        // w^3
  a[3][2] = rot<INV>(a[3][2], -kSqrtHalf, kSqrtHalf); // w^6
  a[3][3] = rot<INV>(a[3][3], -kC1_16, -kS1_16);      // w^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 5) dft5<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
}

// ---------------------------------------------------------------------------
// Stockham iterations with pluggable input and output.
//
// Iteration S of a length-L transform (radix R, Ns = product of the radices
// before it): butterfly j (0 <= j < L/R) of a line reads elements
// j + r L/R, multiplies input r by w_S[k][r] = e^{-+2 pi i r k/(Ns R)}
// (k = j mod Ns), runs the radix-R DFT and writes element
// (j - k) R + k + r Ns.  A work item is butterfly j of a pair of adjacent
// lines (2 cp, 2 cp + 1): its inputs and outputs are 16-byte values holding
// both lines' elements, and its twiddles serve both.  Item b takes
// cp = b mod 4 and j = b / 4, so a warp touches 8 consecutive j of all 8
// lines.  Loaders and storers take (element l, line pair cp) and a float4
// (x, y: line 2 cp; z, w: line 2 cp + 1).

constexpr int kPairs = kT / 2;

__host__ __device__ constexpr int span_before(const RPlan& p, int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= p.r[i];
  return ns;
}

// offset of iteration s in the per-length twiddle table
__host__ __device__ constexpr int tw_offset(const RPlan& p, int s) {
  int off = 0, ns = 1;
  for (int i = 0; i < s; ++i) {
    off += ns * (p.r[i] - 1);
    ns *= p.r[i];
  }
  return off;
}

__host__ __device__ constexpr int tw_table_len(const RPlan& p) { return tw_offset(p, p.nst); }

__device__ __forceinline__ float2 lo2(float4 t) { return make_float2(t.x, t.y); }
__device__ __forceinline__ float2 hi2(float4 t) { return make_float2(t.z, t.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

template <int R, bool INV>
__device__ __forceinline__ void pair_butterfly(float4* t, int k, const float2* tw_row) {
  float2 v0[R], v1[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v0[r] = lo2(t[r]);
    v1[r] = hi2(t[r]);
  }
  if (tw_row != nullptr && k != 0) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw_row[r - 1];
      if (INV) w.y = -w.y;
      v0[r] = cmul(v0[r], w);
      v1[r] = cmul(v1[r], w);
    }
  }
  dft<R, INV>(v0);
  dft<R, INV>(v1);
#pragma unroll
  for (int r = 0; r < R; ++r) t[r] = cat4(v0[r], v1[r]);
}

// compile-time iteration
template <int L, int S, bool INV, class LD, class ST>
__device__ __forceinline__ void iter_ct(const float2* __restrict__ tw, LD&& ld, ST&& st) {
  constexpr RPlan P = rplan(L);
  constexpr int R = P.r[S];
  constexpr int Ns = span_before(P, S);
  constexpr int nbf = L / R;
  constexpr int total = nbf * kPairs;
  constexpr int NB = (total + kThreads - 1) / kThreads;
  constexpr int TO = tw_offset(P, S);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (total % kThreads == 0 || b < total) {
      const int cp = b % kPairs, j = b / kPairs;
      const int k = j % Ns;
      float4 t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = ld(j + r * nbf, cp);
      pair_butterfly<R, INV>(t, k, Ns > 1 ? tw + TO + k * (R - 1) : nullptr);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) st(base + r * Ns, cp, t[r]);
    }
  }
}

// runtime iteration
template <int R, bool INV, class LD, class ST>
__device__ __forceinline__ void iter_rt(const float2* __restrict__ tw, int to, int L, int Ns, LD&& ld, ST&& st) {
  const int nbf = L / R;
  const int total = nbf * kPairs;
  for (int b = threadIdx.x; b < total; b += kThreads) {
    const int cp = b % kPairs, j = b / kPairs;
    const int k = j % Ns;
    float4 t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) t[r] = ld(j + r * nbf, cp);
    pair_butterfly<R, INV>(t, k, tw + to + k * (R - 1));
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st(base + r * Ns, cp, t[r]);
  }
}

struct SmemLd {
  const float2* s;
  __device__ __forceinline__ float4 operator()(int l, int cp) const {
    return reinterpret_cast<const float4*>(s)[l * kPairs + cp];
  }
};
struct SmemSt {
  float2* s;
  __device__ __forceinline__ void operator()(int l, int cp, float4 v) const {
    reinterpret_cast<float4*>(s)[l * kPairs + cp] = v;
  }
};

// Whole transform of kT lines, compile-time length.  ld_first feeds
// iteration 0, st_last takes the last iteration's outputs; the others
// ping-pong between a and b.  Ends with the block synchronised.
template <int L, int S, bool INV, class LD, class ST>
__device__ __forceinline__ void chain_ct(float2* a, float2* b, const float2* tw, LD& ld_first, ST& st_last) {
  constexpr RPlan P = rplan(L);
  constexpr int NST = P.nst;
  if constexpr (P.r[0] == 1) {  // length 1: copy
    for (int cp = threadIdx.x; cp < kPairs; cp += kThreads) st_last(0, cp, ld_first(0, cp));
    __syncthreads();
  } else if constexpr (NST == 1) {
    iter_ct<L, 0, INV>(tw, ld_first, st_last);
    __syncthreads();
  } else if constexpr (S == 0) {
    iter_ct<L, 0, INV>(tw, ld_first, SmemSt{a});
    __syncthreads();
    chain_ct<L, 1, INV>(b, a, tw, ld_first, st_last);
  } else if constexpr (S == NST - 1) {
    // here b holds the previous iteration's output
    iter_ct<L, S, INV>(tw, SmemLd{b}, st_last);
    __syncthreads();
  } else {
    iter_ct<L, S, INV>(tw, SmemLd{b}, SmemSt{a});
    __syncthreads();
    chain_ct<L, S + 1, INV>(b, a, tw, ld_first, st_last);
  }
}

// Iteration 0 split into its loads and its butterflies, so a kernel can
// issue the next tile's loads (into registers) while the current tile runs
// its remaining iterations.  Iteration 0 has Ns = 1: no twiddles.
template <int L>
struct Iter0 {
  static constexpr RPlan P = rplan(L);
  static constexpr int R = P.r[0];
  static constexpr int nbf = L / R;
  static constexpr int total = nbf * kPairs;
  static constexpr int NB = (total + kThreads - 1) / kThreads;
};

template <int L, class LD>
__device__ __forceinline__ void gather0(float4 (&x)[Iter0<L>::NB][Iter0<L>::R], LD& ld) {
  using I = Iter0<L>;
#pragma unroll
  for (int q = 0; q < I::NB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (I::total % kThreads == 0 || b < I::total) {
      const int cp = b % kPairs, j = b / kPairs;
#pragma unroll
      for (int r = 0; r < I::R; ++r) x[q][r] = ld(j + r * I::nbf, cp);
    }
  }
}

template <int L, bool INV, class ST>
__device__ __forceinline__ void butterfly0(float4 (&x)[Iter0<L>::NB][Iter0<L>::R], ST&& st) {
  using I = Iter0<L>;
#pragma unroll
  for (int q = 0; q < I::NB; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (I::total % kThreads == 0 || b < I::total) {
      const int cp = b % kPairs, j = b / kPairs;
      pair_butterfly<I::R, INV>(x[q], 0, nullptr);
#pragma unroll
      for (int r = 0; r < I::R; ++r) st(j * I::R + r, cp, x[q][r]);
    }
  }
}

template <bool INV, class LD, class ST>
__device__ __forceinline__ void iter_rt_dispatch(int R, const float2* tw, int to, int L, int Ns, LD&& ld, ST&& st) {
  switch (R) {
    case 2: iter_rt<2, INV>(tw, to, L, Ns, ld, st); break;
    case 3: iter_rt<3, INV>(tw, to, L, Ns, ld, st); break;
    case 4: iter_rt<4, INV>(tw, to, L, Ns, ld, st); break;
    case 5: iter_rt<5, INV>(tw, to, L, Ns, ld, st); break;
    case 8: iter_rt<8, INV>(tw, to, L, Ns, ld, st); break;
    default:  // radix 1
      for (int idx = threadIdx.x; idx < L * kPairs; idx += kThreads)
        st(idx / kPairs, idx % kPairs, ld(idx / kPairs, idx % kPairs));
  }
}

// Whole transform, runtime length.
template <bool INV, class LD, class ST>
__device__ __forceinline__ void chain_rt(float2* a, float2* b, const float2* tw, const FftLen& f, LD& ld_first,
                                         ST& st_last) {
  int Ns = 1, to = 0;
  for (int i = 0; i < f.nst; ++i) {
    const int R = f.radix[i];
    const bool first = i == 0, last = i == f.nst - 1;
    float2* src = (i & 1) ? a : b;  // output of iteration i - 1
    float2* dst = (i & 1) ? b : a;
    if (first && last) iter_rt_dispatch<INV>(R, tw, to, f.n, Ns, ld_first, st_last);
    else if (first) iter_rt_dispatch<INV>(R, tw, to, f.n, Ns, ld_first, SmemSt{dst});
    else if (last) iter_rt_dispatch<INV>(R, tw, to, f.n, Ns, SmemLd{src}, st_last);
    else iter_rt_dispatch<INV>(R, tw, to, f.n, Ns, SmemLd{src}, SmemSt{dst});
    __syncthreads();
    to += Ns * (R > 1 ? R - 1 : 0);
    Ns *= R;
  }
}

template <int LC, bool INV, class LD, class ST>
__device__ __forceinline__ void transform(float2* a, float2* b, const float2* tw, const FftLen& f, LD& ld_first,
                                          ST& st_last) {
  if constexpr (LC > 0) chain_ct<LC, 0, INV>(a, b, tw, ld_first, st_last);
  else chain_rt<INV>(a, b, tw, f, ld_first, st_last);
}

// Twiddle-table entries of a runtime length.
__device__ __forceinline__ int tw_len_rt(const FftLen& f) {
  int off = 0, ns = 1;
  for (int i = 0; i < f.nst; ++i) {
    off += ns * (f.radix[i] > 1 ? f.radix[i] - 1 : 0);
    ns *= f.radix[i];
  }
  return off;
}

// Pruning of the 512-point strided passes by a box {x0, x1, y0, y1, z0, z1}:
// kPrunePlanes: the view's outer index is o = s nz + z (nz planes per shell)
// and only the planes z0 <= z <= z1 are transformed; kPruneOutY: only the
// rows y0..y1 are written; kPruneInY / kPruneInZ: rows outside y0..y1 /
// z0..z1 are zeros of the input and are not read.
constexpr int kPrunePlanes = 1, kPruneOutY = 2, kPruneInY = 4, kPruneInZ = 8;

// A strided-axis view: element (o, l, i) at o*so + l*sl + i, l in [0, L),
// i in [0, inner); a tile is one o and kT consecutive i.
struct StridedView {
  int64_t sl, so;
  int inner;
  int64_t n_outer;
};

struct StridedTile {
  const float2* in;
  float2* out;
  int64_t sl;
  int valid;  // columns of this tile inside [0, inner): 4 or 8 (inner is a multiple of 4)
  __device__ __forceinline__ float4 operator()(int l, int cp) const {
    return 2 * cp < valid ? __ldcg(reinterpret_cast<const float4*>(in + (int64_t)l * sl + 2 * cp))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ __forceinline__ void operator()(int l, int cp, float4 v) const {
    if (2 * cp < valid) *reinterpret_cast<float4*>(out + (int64_t)l * sl + 2 * cp) = v;
  }
};

__device__ __forceinline__ StridedTile strided_tile(const float2* in, float2* out, const StridedView& v,
                                                    int64_t tile) {
  const int tpo = (v.inner + kT - 1) / kT;
  const int64_t o = tile / tpo;
  const int i0 = (int)(tile - o * tpo) * kT;
  return StridedTile{in + o * v.so + i0, out + o * v.so + i0, v.sl, min(kT, v.inner - i0)};
}

// ---------------------------------------------------------------------------
// kernels

// Strided-axis transform (in place allowed: a tile's reads all happen in the
// first iteration, before the barrier that precedes its writes).
// Tile of a strided view staged into shared memory (column layout) with
// 16-byte cp.async copies; columns past the view's end are zero-filled.
__device__ __forceinline__ void stage_strided_tile(float2* s, const float2* in, const StridedView& v, int L,
                                                   int64_t tile) {
  const int tpo = (v.inner + kT - 1) / kT;
  const int64_t o = tile / tpo;
  const int i0 = (int)(tile - o * tpo) * kT;
  const float2* base = in + o * v.so + i0;
  for (int idx = threadIdx.x; idx < L * kPairs; idx += kThreads) {
    const int l = idx / kPairs, cp = idx % kPairs;
    const bool ok = i0 + 2 * cp < v.inner;
    cp_async16(s + l * kT + 2 * cp, ok ? base + (int64_t)l * v.sl + 2 * cp : in, ok);
  }
}

// Strided-axis transform (in place allowed: a tile is read, through the
// staging copy, before any of its elements is written).  Persistent CTAs
// stage the next tile with cp.async while the current one is transformed;
// iteration 0 reads the staged tile, the iterations ping-pong between the
// work buffer and the staged tile's buffer, and the last one stores to
// global memory.
template <int LC, bool INV>
__global__ void __launch_bounds__(kThreads, LC > 0 ? 2 : 1)
    strided_kernel(const float2* in, float2* out, StridedView v, FftLen f, const float2* __restrict__ stw) {
  extern __shared__ float4 smem4[];
  const int L = LC > 0 ? LC : f.n;
  float2* p0 = reinterpret_cast<float2*>(smem4);
  float2* p1 = p0 + L * kT;
  float2* w = p1 + L * kT;
  float2* tws = w + L * kT;
  const int ntw = LC > 0 ? tw_table_len(rplan(LC)) : tw_len_rt(f);
  for (int i = threadIdx.x; i < ntw; i += kThreads) tws[i] = __ldg(stw + i);
  const int64_t ntiles = v.n_outer * ((v.inner + kT - 1) / kT);
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  stage_strided_tile(p0, in, v, L, t);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it) {
    const int64_t tn = t + gridDim.x;
    float2* cur = (it & 1) ? p1 : p0;
    if (tn < ntiles) stage_strided_tile((it & 1) ? p0 : p1, in, v, L, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    StridedTile io = strided_tile(in, out, v, t);
    SmemLd ld{cur};
    // iteration 0 writes w, then the chain alternates w <-> cur
    transform<LC, INV>(w, cur, tws, f, ld, io);
    t = tn;
  }
}

// Kernel spectra for the fused multiply: the octant K^_s[kzf][kyf][kx] with
// rows padded to the spectrum pitch px (zeros for kx > n[0]/2).  Element
// (kz, i) of the z pass, i = ky * px + kx, uses (min(kz, nz-kz),
// min(ky, ny-ky), kx).
struct KhatArgs {
  const float* khat;  // octant of shell 0 (nullptr: multiply by 1)
  int64_t shell_stride;
  int px, ny, nz, oy;
};

// Inverse z pass of every shell at once: a half-spectrum tile is staged in
// shared memory once, then for each shell s the first iteration reads it
// multiplied by K^_s (Eq. 9 in Fourier space) and the last writes the
// z-transformed product to that shell's scratch spectrum out + s * out_stride.
// The tile's slab of K^_s (nz/2 + 1 rows of kT values) is fetched with
// cp.async while the previous shell finishes.  khat == nullptr: one
// transform, factor 1.
template <int LC>
__global__ void __launch_bounds__(kThreads, 2)
    zmulti_kernel(const float2* in, float2* out, int64_t out_stride, int nshells, StridedView v, FftLen f,
                  const float2* __restrict__ stw, KhatArgs K) {
  extern __shared__ float4 smem4[];
  const int L = LC > 0 ? LC : f.n;
  const int OZ = L / 2 + 1;
  float2* pristine = reinterpret_cast<float2*>(smem4);
  float2* a = pristine + L * kT;
  float2* b = a + L * kT;
  float2* tws = b + L * kT;
  const int ntw = LC > 0 ? tw_table_len(rplan(LC)) : tw_len_rt(f);
  float* slab = reinterpret_cast<float*>(tws + ((ntw + 1) & ~1));
  for (int i = threadIdx.x; i < ntw; i += kThreads) tws[i] = __ldg(stw + i);
  const int64_t ntiles = (v.inner + kT - 1) / kT;
  // two halves of 4 columns per tile: px is a multiple of 4 and i0 of 8, so
  // each half lies in one ky row of the spectrum
  auto load_slab = [&](int s, int64_t tile) {
    const float* kh = K.khat + (int64_t)s * K.shell_stride;
    for (int idx = threadIdx.x; idx < 2 * OZ; idx += kThreads) {
      const int kzf = idx >> 1, h = idx & 1;
      const int i = (int)tile * kT + 4 * h;
      const bool ok = i < v.inner;
      const int ky = i / K.px, kx = i - (i / K.px) * K.px;
      const int kyf = min(ky, K.ny - ky);
      cp_async16(slab + kzf * kT + 4 * h, ok ? kh + ((int64_t)kzf * K.oy + kyf) * K.px + kx : K.khat, ok);
    }
  };
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (int)t * kT;
    const int valid = min(kT, v.inner - i0);
    for (int idx = threadIdx.x; idx < L * (kT / 2); idx += kThreads) {
      const int l = idx / (kT / 2), c = (idx % (kT / 2)) * 2;
      const bool ok = c < valid;
      cp_async16(pristine + l * kT + c, ok ? in + (int64_t)l * v.sl + i0 + c : in, ok);
    }
    if (K.khat) load_slab(0, t);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int s = 0; s < nshells; ++s) {
      const bool mul = K.khat != nullptr;
      auto ld = [&](int l, int cp) {
        const float4 x = reinterpret_cast<const float4*>(pristine)[l * kPairs + cp];
        if (!mul) return x;
        const float2 m = reinterpret_cast<const float2*>(slab)[min(l, L - l) * kPairs + cp];
        return make_float4(x.x * m.x, x.y * m.x, x.z * m.y, x.w * m.y);
      };
      StridedTile st{nullptr, out + (int64_t)s * out_stride + i0, v.sl, valid};
      if constexpr (LC > 0) {
        constexpr RPlan P = rplan(LC);
        static_assert(P.nst >= 2, "the multi-shell z pass needs two or more iterations");
        iter_ct<LC, 0, true>(tws, ld, SmemSt{a});
        __syncthreads();
        // the slab of shell s has been consumed: fetch the next shell's
        if (mul && s + 1 < nshells) load_slab(s + 1, t);
        cp_async_commit();
        chain_ct<LC, 1, true>(b, a, tws, ld, st);
      } else {
        chain_rt<true>(a, b, tws, f, ld, st);
        if (mul && s + 1 < nshells) load_slab(s + 1, t);
        cp_async_commit();
      }
      cp_async_wait<0>();
      __syncthreads();
    }
  }
}

// x-pass tiles: kT rows of one axis line each.  Loads, the even/odd
// (un)packing and stores map consecutive threads to consecutive rows first.

// Forward x pass: real rows of length nx = 2M -> half-spectrum rows (pitch
// px).  z[m] = x[2m] + i x[2m+1], Z = DFT_M(z), then X[k] = E[k] +
// e^{-2 pi i k/nx} O[k], E = (Z[k] + conj Z[M-k]) / 2,
// O = (Z[k] - conj Z[M-k]) / 2i, k = 0..M.  The transform's first iteration
// reads the real rows from global memory; its output stays in shared memory
// for the split.
// box (null: every row): the rows (y, z) of the box {x0, x1, y0, y1, z0, z1}
// alone, the field being zero elsewhere; the other rows are not written.
template <int MC>
__global__ void __launch_bounds__(kThreads, min_blocks(MC))
    x_r2c_kernel(const float* __restrict__ in, float2* __restrict__ out, int nx, int px, int64_t rows, FftLen f,
                 const float2* __restrict__ stw, const float2* __restrict__ tw, const int* __restrict__ box, int ny) {
  extern __shared__ float4 smem4[];
  const int M = MC > 0 ? MC : nx / 2;
  const int NX = 2 * M;
  float2* a = reinterpret_cast<float2*>(smem4);
  float2* b = a + M * kT;
  float2* tws = b + M * kT;
  const int ntw = MC > 0 ? tw_table_len(rplan(MC)) : tw_len_rt(f);
  float2* twn = tws + ntw;
  for (int i = threadIdx.x; i < ntw; i += kThreads) tws[i] = __ldg(stw + i);
  for (int i = threadIdx.x; i <= M; i += kThreads) twn[i] = __ldg(tw + i);
  __syncthreads();
  // visited rows: every row, or the box's (y0..y1, z0..z1) in order
  int64_t y0 = 0, nyb = ny > 0 ? ny : 1, z0 = 0, count = rows;
  if (box) {
    y0 = box[2];
    nyb = box_len(box[2], box[3]);
    z0 = box[4];
    const int64_t nzb = box_len(box[4], box[5]);
    count = nyb > 0 && nzb > 0 ? nyb * nzb : 0;
    if (nyb <= 0) nyb = 1;
  }
  auto row_of = [=](int64_t c) { return box ? (z0 + c / nyb) * ny + y0 + c % nyb : c; };
  const int64_t ntiles = (count + kT - 1) / kT;
  auto rows_ld = [&](int64_t tile) {
    const int64_t r0 = tile * kT;
    const int valid = (int)(count - r0 < kT ? count - r0 : kT);
    return [=](int m, int cp) {
      const int c = 2 * cp;
      const float2 z0v = c < valid ? __ldg(reinterpret_cast<const float2*>(in + row_of(r0 + c) * NX) + m)
                                   : make_float2(0.f, 0.f);
      const float2 z1v = c + 1 < valid ? __ldg(reinterpret_cast<const float2*>(in + row_of(r0 + c + 1) * NX) + m)
                                       : make_float2(0.f, 0.f);
      return cat4(z0v, z1v);
    };
  };
  // the transform's output buffer: not the one its last iteration reads
  float2* res = nullptr;
  if constexpr (MC > 0) res = (rplan(MC).nst % 2 == 1) ? a : b;
  else res = (f.nst % 2 == 1) ? a : b;
  auto split = [&](int64_t t) {
    const int64_t r0 = t * kT;
    const int valid = (int)(count - r0 < kT ? count - r0 : kT);
    const float2* s = res;
    for (int idx = threadIdx.x; idx < kT * px; idx += kThreads) {
      const int c = idx % kT, k = idx / kT;
      if (c >= valid) continue;
      float2 X = make_float2(0.f, 0.f);
      if (k <= M) {
        const float2 zk = s[(k == M ? 0 : k) * kT + c];
        const float2 zc = cconj(s[(k == 0 ? 0 : M - k) * kT + c]);
        const float2 E = cscale(cadd(zk, zc), 0.5f);
        const float2 O = cscale(cmul_mi<false>(csub(zk, zc)), 0.5f);
        X = cadd(E, cmul(twn[k], O));
      }
      out[row_of(r0 + c) * px + k] = X;
    }
    __syncthreads();
  };
  if constexpr (MC > 0 && rplan(MC).nst >= 2) {
    float4 x[Iter0<MC>::NB][Iter0<MC>::R];
    int64_t t = blockIdx.x;
    if (t < ntiles) {
      auto ld = rows_ld(t);
      gather0<MC>(x, ld);
    }
    for (; t < ntiles; t += gridDim.x) {
      butterfly0<MC, false>(x, SmemSt{a});
      __syncthreads();
      const int64_t tn = t + gridDim.x;
      if (tn < ntiles) {
        auto ld = rows_ld(tn);
        gather0<MC>(x, ld);
      }
      SmemSt st{res};
      auto unused = rows_ld(t);
      chain_ct<MC, 1, false>(b, a, tws, unused, st);
      split(t);
    }
  } else {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      auto ld = rows_ld(t);
      SmemSt st{res};
      transform<MC, false>(a, b, tws, f, ld, st);
      split(t);
    }
  }
}

struct RealRowsOut {
  float* out;
  int nx;
  int valid;
  __device__ __forceinline__ void operator()(int m, int cp, float4 v) const {
    const int c = 2 * cp;
    if (c < valid) *reinterpret_cast<float2*>(out + (int64_t)c * nx + 2 * m) = lo2(v);
    if (c + 1 < valid) *reinterpret_cast<float2*>(out + (int64_t)(c + 1) * nx + 2 * m) = hi2(v);
  }
};

// Inverse x pass: half-spectrum rows -> real rows.  Persistent CTAs stage
// the next tile's rows (X[0..M], row pitch M + 2) with 16-byte cp.async
// copies while the current tile is unpacked into Z (pairs (k, M-k)),
// transformed (z = IDFT_M(Z), unnormalised) and written by the last
// iteration as x[2m] = Re z[m], x[2m+1] = Im z[m].  Input rows are contiguous
// (pitch px); output row r goes to
// out + (r / rows_per_shell) * out_shell_stride + (r % rows_per_shell) * nx.
// Even, so that every staged row starts on a 16-byte boundary (odd M too).
__host__ __device__ constexpr int stage_pitch(int M) { return (M + 3) / 2 * 2; }

template <int MC>
__global__ void __launch_bounds__(kThreads, min_blocks(MC))
    x_c2r_kernel(const float2* __restrict__ in, float* __restrict__ out, int nx, int px, int64_t rows,
                 int64_t rows_per_shell, int64_t out_shell_stride, FftLen f, const float2* __restrict__ stw,
                 const float2* __restrict__ tw, const int* __restrict__ box, int ny) {
  extern __shared__ float4 smem4[];
  const int M = MC > 0 ? MC : nx / 2;
  const int NX = 2 * M;
  const int LP = stage_pitch(M);
  float2* s0 = reinterpret_cast<float2*>(smem4);
  float2* s1 = s0 + kT * LP;
  float2* u = s1 + kT * LP;
  float2* w = u + (M + 1) * kT;
  float2* tws = w + (M + 1) * kT;
  const int ntw = MC > 0 ? tw_table_len(rplan(MC)) : tw_len_rt(f);
  float2* twn = tws + ntw;
  for (int i = threadIdx.x; i < ntw; i += kThreads) tws[i] = __ldg(stw + i);
  for (int i = threadIdx.x; i <= M; i += kThreads) twn[i] = __ldg(tw + i);
  // visited rows: every row, or (box) the rows of the planes box[4] ..
  // box[5] of every shell, numbered q = shell * nrb + row in those planes
  int64_t count = rows, nrb = rows_per_shell, rb0 = 0;
  if (box) {
    nrb = (int64_t)box_len(box[4], box[5]) * ny;
    rb0 = (int64_t)box[4] * ny;
    count = (rows / rows_per_shell) * nrb;
  }
  auto row_of = [&](int64_t q) -> int64_t {  // the row's index in [shell][rows_per_shell]
    if (!box) return q;
    const int64_t sh = q / nrb;
    return sh * rows_per_shell + rb0 + (q - sh * nrb);
  };
  const int64_t ntiles = (count + kT - 1) / kT;
  // X[0..M] as pairs (k, k+1), k even: M/2 + 1 copies per row; for even M
  // the last pair also reads padding column M + 1 (< px)
  const int np = M / 2 + 1;
  auto stage = [&](float2* s, int64_t tile) {
    const int64_t r0 = tile * kT;
    for (int idx = threadIdx.x; idx < kT * np; idx += kThreads) {
      const int c = idx / np, k = 2 * (idx - c * np);
      const bool ok = r0 + c < count;
      cp_async16(s + c * LP + k, ok ? (const void*)(in + row_of(r0 + c) * px + k) : (const void*)in, ok);
    }
  };
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  stage(s0, t);
  cp_async_commit();
  const int half = M / 2 + 1;
  for (int it = 0; t < ntiles; ++it) {
    const int64_t tn = t + gridDim.x;
    const float2* sc = (it & 1) ? s1 : s0;
    if (tn < ntiles) stage((it & 1) ? s0 : s1, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int64_t r0 = t * kT;
    const int valid = (int)(count - r0 < kT ? count - r0 : kT);
    // unpack: Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k])
    for (int idx = threadIdx.x; idx < kT * half; idx += kThreads) {
      const int c = idx % kT, k = idx / kT;
      const float2 a = sc[c * LP + k], b = sc[c * LP + M - k];
      const float2 ca = cconj(a), cb = cconj(b);
      u[k * kT + c] = cadd(cadd(a, cb), cmul_mi<true>(cmul(cconj(twn[k]), csub(a, cb))));
      if (k != 0 && 2 * k != M)
        u[(M - k) * kT + c] = cadd(cadd(b, ca), cmul_mi<true>(cmul(cconj(twn[M - k]), csub(b, ca))));
    }
    __syncthreads();
    SmemLd ld{u};
    // rows of this tile may belong to two shells (or leave the box's
    // planes): split the output per row
    const int64_t f0 = row_of(r0);
    const int64_t sh0 = f0 / rows_per_shell;
    const int64_t rr0 = f0 - sh0 * rows_per_shell;
    if (box ? (r0 % nrb) + valid <= nrb : rr0 + valid <= rows_per_shell) {
      RealRowsOut st{out + sh0 * out_shell_stride + rr0 * NX, NX, valid};
      transform<MC, true>(w, u, tws, f, ld, st);
    } else {
      auto st = [&](int m, int cp, float4 v) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * cp + h;
          if (c >= valid) continue;
          const int64_t row = row_of(r0 + c), sh = row / rows_per_shell, rr = row - sh * rows_per_shell;
          *reinterpret_cast<float2*>(out + sh * out_shell_stride + rr * NX + 2 * m) = h ? hi2(v) : lo2(v);
        }
      };
      transform<MC, true>(w, u, tws, f, ld, st);
    }
    t = tn;
  }
}

// shared-memory bytes of each kernel
inline size_t strided_smem(int L) { return ((size_t)3 * L * kT + L) * sizeof(float2); }
inline size_t zmulti_smem(int L) {
  return ((size_t)3 * L * kT + L + 2) * sizeof(float2) + (size_t)(L / 2 + 1) * kT * sizeof(float);
}
inline size_t xpass_smem(int nx) {
  return ((size_t)2 * kT * stage_pitch(nx / 2) + (size_t)2 * kT * (nx / 2 + 1) + nx + 2) * sizeof(float2);
}

// Launch helpers (one translation unit each; they pick the compile-time
// length when LC/MC is one of the instantiated lengths).
// cols: columns per tile of the 512-point register kernels (8 or 16)
// box (device, may be null; 512-point axes only) with `mode` (the pruning
// bits of ck_fft_sreg.cuh: transform only the box's planes, write only its
// rows y, read only its rows y or z as nonzero input); for the z pass with
// the multiply, only the box's planes are written.  launch_zmulti's tw: for
// L = 512 the twiddle matrix w512^(l2 m1) at [m1 * 32 + l2] (Plan::twm),
// unused otherwise.
void launch_strided(int L, bool inv, const float2* in, float2* out, const StridedView& v, const FftLen& f,
                    const float2* stw, const float2* tw, int cols, int sm_count, cudaStream_t st,
                    const int* box = nullptr, int nz = 0, int mode = 0);
void launch_zmulti(int L, const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                   const FftLen& f, const float2* stw, const float2* tw, const KhatArgs& K, int sm_count,
                   cudaStream_t st, const int* box = nullptr, int cols = 8);
// box (device, may be null): the input is zero outside the box; only its rows
// (ny rows per plane) are transformed and written.
void launch_x_r2c(int M, const float* in, float2* out, int nx, int px, int64_t rows, const FftLen& f,
                  const float2* stw, const float2* tw, int sm_count, cudaStream_t st, const int* box = nullptr,
                  int ny = 0);
// The forward x pass of 512-cell rows in registers (ck_fft_xr.cu): the same
// arguments for M = 256 (tw: e^{-2 pi i t / 512}).
void launch_xr2c_reg(const float* in, float2* out, int px, int64_t rows, const float2* tw, int sm_count,
                     cudaStream_t st, const int* box, int ny);
// The inverse x pass of 512-cell rows in registers: launch_x_c2r's arguments
// for M = 256 and px = 260.
void launch_xc2r_reg(const float2* in, float* out, int px, int64_t rows, int64_t rows_per_shell,
                     int64_t out_shell_stride, const float2* tw, int sm_count, cudaStream_t st, const int* box,
                     int ny);
// box (device, may be null): only the rows of the planes box[4] .. box[5]
// (ny rows per plane) of every shell are transformed and written.
void launch_x_c2r(int M, const float2* in, float* out, int nx, int px, int64_t rows, int64_t rows_per_shell,
                  int64_t out_shell_stride, const FftLen& f, const float2* stw, const float2* tw, int sm_count,
                  cudaStream_t st, const int* box = nullptr, int ny = 0);

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
