// ck_fft_sreg.cuh -- 512-point transforms along a strided axis (y or z)
// with the butterflies in registers, for the passes of Sec. 2.4's FFT
// convolution on 512-cell axes.
//
// A tile is C adjacent columns (C = 8 or 16) x 512 rows of a strided view,
// staged in shared memory as S[row][c]; a CTA has 32 C threads.  With
// l = 32 l1 + l2 and m = m1 + 16 m2,
//   X[m1 + 16 m2] = sum_l2 w32^(l2 m2) w512^(l2 m1) sum_l1 w16^(l1 m1) x[32 l1 + l2]
// (w_n = e^{-+2 pi i / n}).  Step A: thread (c, l2) runs the 16-point DFT
// over l1 and applies w512^(l2 m1), writing the padded transpose T.  Step
// B: threads (c, m1, h) take the even (h = 0) or odd (h = 1) l2 of column
// m1 of T and run a 16-point DFT (E or O); one exchange with the partner
// lane (lane ^ C) gives each thread half of
// X[m1 + 16 k] = E[k] + w32^k O[k] and X[m1 + 16 (k + 16)] = E[k] - w32^k O[k],
// which go straight to global memory (C columns = 8 C contiguous bytes).
//
// sreg512_kernel: one transform per tile, double-buffered staging (in
// place allowed); optionally only the planes and rows of a box.
// zreg512_kernel: the first inverse pass of Eqs. 9-10: the spectrum tile is
// staged once and, for every shell s, multiplied by the tile's slab of K^_s
// while step A reads it; outputs go to out + s * stride.
#pragma once

#include "ck_fft_core.cuh"

namespace ck {
namespace fft {

template <int C>
struct Sreg {
  static_assert(C == 8 || C == 16, "tile widths");
  static constexpr int L = 512, P = 16, Q = 32;
  static constexpr int NT = 32 * C;       // threads per CTA
  static constexpr int TPAD = P * C + 8;  // float2 per l2 row of T (conflict-free half-warps)
  static constexpr size_t s_bytes = (size_t)L * C * sizeof(float2);
  static constexpr size_t t_bytes = (size_t)Q * TPAD * sizeof(float2);
  static constexpr size_t twa_bytes = (size_t)Q * (P + 1) * sizeof(float2);  // w512^(l2 m1), row pitch 17
  static constexpr size_t slab_bytes = (size_t)(L / 2 + 1) * C * sizeof(float);
  // plain: S0 S1 T twa; multi-shell: S slab T (its step A reads the
  // twiddles from the global table, which keeps three 8-column CTAs per SM)
  static constexpr size_t plain_bytes = 2 * s_bytes + t_bytes + twa_bytes;
  static constexpr size_t multi_bytes = s_bytes + slab_bytes + t_bytes;
};

// Twiddle table twa[l2][m1] = w512^(l2 m1) from the axis table
// tw[t] = e^{-2 pi i t / 512} (conjugated for INV).
template <int C, bool INV>
__device__ __forceinline__ void sreg_tables(float2* twa, const float2* __restrict__ tw) {
  using S = Sreg<C>;
  for (int i = threadIdx.x; i < S::Q * S::P; i += S::NT) {
    const int l2 = i / S::P, m1 = i - l2 * S::P;
    const float2 w = __ldg(tw + l2 * m1);
    twa[l2 * (S::P + 1) + m1] = INV ? cconj(w) : w;
  }
}

// Step A for thread (c, l2); ld(l1) returns x[32 l1 + l2] of column c (times
// K^ in the multi-shell pass), w(m1) the twiddle w512^(l2 m1).
template <int C, bool INV, class LD, class TW>
__device__ __forceinline__ void sreg_step_a(float2* T, int c, int l2, LD&& ld, TW&& w) {
  using S = Sreg<C>;
  float2 v[S::P];
#pragma unroll
  for (int l1 = 0; l1 < S::P; ++l1) v[l1] = ld(l1);
  dft16<INV>(v);
  float2* tr = T + l2 * S::TPAD + c;
  tr[0] = v[0];
#pragma unroll
  for (int m1 = 1; m1 < S::P; ++m1) tr[m1 * C] = cmul(v[m1], w(m1));
}

// cos and sin of 2 pi k / 32, k < 8 (folded to immediates in unrolled loops)
__host__ __device__ constexpr float cos32(int k) {
  return k == 0 ? 1.0f
       : k == 1 ? 0.98078528040323044913f
       : k == 2 ? 0.92387953251128675613f
       : k == 3 ? 0.83146961230254523708f
       : k == 4 ? 0.70710678118654752440f
       : k == 5 ? 0.55557023301960222474f
       : k == 6 ? 0.38268343236508977173f
       : 0.19509032201612826785f;
}
__host__ __device__ constexpr float sin32(int k) { return cos32(8 - k); }

// Rows thread (m1, h) of step B writes: bit k for row m1 + 128 h + 16 k and
// bit k + 8 for that row + 256 (k < 8), set where rlo <= row <= rhi.
__device__ __forceinline__ uint32_t sreg_row_mask(int m1, int h, int rlo, int rhi) {
  uint32_t mask = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int row = m1 + 128 * h + 16 * k;
    if (row >= rlo && row <= rhi) mask |= 1u << k;
    if (row + 256 >= rlo && row + 256 <= rhi) mask |= 1u << (k + 8);
  }
  return mask;
}

// Step B for thread (c, m1, h), lane bit log2(C) = h: the 16-point DFT of
// the even (h = 0: E) or odd (h = 1: O) l2, then one exchange with the
// partner lane gives thread h the pairs k + 8 h (k < 8):
// X[m1 + 16 kk] = E[kk] + w32^kk O[kk] and X[m1 + 16 (kk + 16)] = E[kk] - w32^kk O[kk],
// kk = k + 8 h.  w32^(k + 8) = w32^k w32^8 (w32^8 = -+i), so both halves
// multiply by the same compile-time w32^k and h = 1 rotates by w32^8.
// Row m1 + 16 kk goes to col[row * sl] where bit k (and k + 8 for the
// second row) of mask is set.
template <int C, bool INV>
__device__ __forceinline__ void sreg_step_b(const float2* T, int c, int m1, int h, float2* col, int64_t sl,
                                            uint32_t mask) {
  using S = Sreg<C>;
  float2 y[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) y[j] = T[(2 * j + h) * S::TPAD + m1 * C + c];
  dft16<INV>(y);
  float2* p = col + (int64_t)(m1 + 128 * h) * sl;  // row m1 + 16 kk for k = 0
  const int64_t s16 = 16 * sl, s256 = 256 * sl;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    // h = 0 sends E[k + 8] and keeps E[k]; h = 1 sends O[k] and keeps O[k + 8]
    const float2 send = h ? y[k] : y[k + 8];
    float2 recv;
    recv.x = __shfl_xor_sync(0xFFFFFFFFu, send.x, C);
    recv.y = __shfl_xor_sync(0xFFFFFFFFu, send.y, C);
    const float2 a = h ? recv : y[k];
    const float2 z = h ? y[k + 8] : recv;
    const float2 wz = k == 0 ? z : rot<INV>(z, cos32(k), sin32(k));
    const float2 b = h ? cmul_mi<INV>(wz) : wz;
    if (mask & (1u << k)) p[0] = cadd(a, b);
    if (mask & (1u << (k + 8))) p[s256] = csub(a, b);
    p += s16;
  }
}

// The tile of outer index o and first column i0 of a strided view (C
// columns x 512 rows) into S[row][c] with 16-byte cp.async copies; columns
// past the view's end, and rows outside [rlo, rhi] (known zeros), are
// zero-filled.
template <int C>
__device__ __forceinline__ void sreg_stage(float2* s, const float2* in, const StridedView& v, int64_t o, int i0,
                                           int rlo = 0, int rhi = 511) {
  using S = Sreg<C>;
  const float2* base = in + o * v.so + i0;
  for (int idx = threadIdx.x; idx < S::L * (C / 2); idx += S::NT) {
    const int l = idx / (C / 2), cp = idx % (C / 2);
    const bool ok = i0 + 2 * cp < v.inner && l >= rlo && l <= rhi;
    cp_async16(s + l * C + 2 * cp, ok ? base + (int64_t)l * v.sl + 2 * cp : in, ok);
  }
}

// Pruning by a box {x0, x1, y0, y1, z0, z1} (null: none) with the mode bits
// of ck_fft_core.cuh (kPrunePlanes, kPruneOutY, kPruneInY, kPruneInZ).
template <int C, bool INV>
__global__ void __launch_bounds__(Sreg<C>::NT, C == 8 ? 2 : 1)
    sreg512_kernel(const float2* in, float2* out, StridedView v, const float2* __restrict__ tw,
                   const int* __restrict__ box, int nz, int mode) {
  using S = Sreg<C>;
  extern __shared__ float4 smem4[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
  float2* T = reinterpret_cast<float2*>(sm + 2 * S::s_bytes);
  float2* twa = reinterpret_cast<float2*>(sm + 2 * S::s_bytes + S::t_bytes);
  auto sbuf = [&](int b) { return reinterpret_cast<float2*>(sm + b * S::s_bytes); };
  sreg_tables<C, INV>(twa, tw);
  const int tid = threadIdx.x;
  const int ca = tid % C, l2 = tid / C;                                // step A
  const int cb = tid % C, hb = (tid / C) & 1, m1 = tid / (2 * C);      // step B
  const int tpo = (v.inner + C - 1) / C;
  if (!box) mode = 0;
  const bool planes = (mode & kPrunePlanes) != 0;
  int zlo = 0, nzb = nz, rlo = 0, rhi = S::L - 1, ilo = 0, ihi = S::L - 1;
  if (planes) {
    zlo = box[4];
    nzb = box_len(box[4], box[5]);
  }
  if (mode & kPruneOutY) {
    rlo = box[2];
    rhi = box[3];
  }
  if (mode & kPruneInY) {
    ilo = box[2];
    ihi = box[3];
  } else if (mode & kPruneInZ) {
    ilo = box[4];
    ihi = box[5];
  }
  const int64_t outers = planes ? (v.n_outer / nz) * nzb : v.n_outer;
  const int64_t ntiles = outers * tpo;
  const uint32_t rmask = sreg_row_mask(m1, hb, rlo, rhi);
  // tile -> outer index of the view (plane zlo + .. of a shell) and first column
  auto outer_of = [&](int64_t tile) {
    const int64_t ot = tile / tpo;
    return planes ? (ot / nzb) * nz + zlo + ot % nzb : ot;
  };
  auto col_of = [&](int64_t tile) { return (int)(tile % tpo) * C; };
  int64_t t = blockIdx.x;
  if (t < ntiles) sreg_stage<C>(sbuf(0), in, v, outer_of(t), col_of(t), ilo, ihi);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it) {
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) sreg_stage<C>(sbuf((it + 1) & 1), in, v, outer_of(tn), col_of(tn), ilo, ihi);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float2* cur = sbuf(it & 1);
    const float2* cc = cur + l2 * C + ca;
    const float2* tk = twa + l2 * (S::P + 1);
    sreg_step_a<C, INV>(T, ca, l2, [&](int l1) { return cc[S::Q * l1 * C]; }, [&](int m1) { return tk[m1]; });
    __syncthreads();
    const int64_t o = outer_of(t);
    const int i0 = col_of(t);
    sreg_step_b<C, INV>(T, cb, m1, hb, out + o * v.so + i0 + cb, v.sl, i0 + cb < v.inner ? rmask : 0u);
    t = tn;
  }
}

template <int C>
__global__ void __launch_bounds__(Sreg<C>::NT, C == 8 ? 3 : 1)
    zreg512_kernel(const float2* in, float2* out, int64_t out_stride, int nshells, StridedView v,
                   const float2* __restrict__ twm, KhatArgs K, const int* __restrict__ box) {
  using S = Sreg<C>;
  constexpr int OZ = S::L / 2 + 1;
  extern __shared__ float4 smem4[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
  float2* Sx = reinterpret_cast<float2*>(sm);
  float* slab = reinterpret_cast<float*>(sm + S::s_bytes);
  float2* T = reinterpret_cast<float2*>(sm + S::s_bytes + S::slab_bytes);
  const int tid = threadIdx.x;
  const int ca = tid % C, l2 = tid / C;
  const int cb = tid % C, hb = (tid / C) & 1, m1 = tid / (2 * C);
  const int64_t ntiles = (v.inner + C - 1) / C;
  const bool mul = K.khat != nullptr;
  // box (null: none): only the output rows (kz -> z) box[4] .. box[5] are written
  const uint32_t rmask = sreg_row_mask(m1, hb, box ? box[4] : 0, box ? box[5] : S::L - 1);
  // C / 4 groups of 4 columns per tile: px is a multiple of 4 and i0 of C,
  // so each group lies in one ky row of the spectrum.  A thread copies only
  // group h = tid mod (C / 4) (NT is a multiple of C / 4), whose offset in
  // an octant plane, kyf px + kx (-1: past the spectrum), is the same for
  // every shell and is computed once per tile.
  const int hs = tid % (C / 4);
  const int64_t oplane = (int64_t)K.oy * K.px;
  auto slab_offset = [&](int64_t tile) {
    const int i = (int)tile * C + 4 * hs;
    if (i >= v.inner) return -1;
    const int ky = i / K.px, kx = i - ky * K.px;
    return min(ky, K.ny - ky) * K.px + kx;
  };
  auto load_slab = [&](int s, int off) {
    const float* kh = K.khat + (int64_t)s * K.shell_stride + (off < 0 ? 0 : off);
    for (int idx = tid; idx < (C / 4) * OZ; idx += S::NT) {
      const int kzf = idx / (C / 4);
      cp_async16(slab + kzf * C + 4 * hs, off >= 0 ? kh + kzf * oplane : K.khat, off >= 0);
    }
  };
  auto stage = [&](int64_t tile) {
    const int i0 = (int)tile * C;
    for (int idx = tid; idx < S::L * (C / 2); idx += S::NT) {
      const int l = idx / (C / 2), c = (idx % (C / 2)) * 2;
      const bool ok = i0 + c < v.inner;
      cp_async16(Sx + l * C + c, ok ? in + (int64_t)l * v.sl + i0 + c : in, ok);
    }
  };
  // K^ is even in ky, so the tiles of rows ky and ny - ky read the same
  // slabs: visit tiles from both ends in turn (schedule index j -> tile),
  // so that the second reader of a slab finds it in L2
  auto tile_of = [&](int64_t j) { return (j & 1) ? ntiles - 1 - (j >> 1) : (j >> 1); };
  int64_t j = blockIdx.x;
  int off = j < ntiles && mul ? slab_offset(tile_of(j)) : -1;
  if (j < ntiles) {
    stage(tile_of(j));
    if (mul) load_slab(0, off);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  for (; j < ntiles; j += gridDim.x) {
    const int64_t t = tile_of(j);
    const int i0 = (int)t * C;
    const int64_t jn = j + gridDim.x;
    const int64_t tn = jn < ntiles ? tile_of(jn) : ntiles;
    const int off_next = tn < ntiles && mul ? slab_offset(tn) : -1;
    for (int s = 0; s < nshells; ++s) {
      // K^ depends on min(kz, 512 - kz): kz = 32 l1 + l2 for l1 < 8, 512 - kz beyond
      const float2* xc = Sx + l2 * C + ca;
      const float* sa = slab + l2 * C + ca;
      sreg_step_a<C, true>(
          T, ca, l2,
          [&](int l1) {
            const float2 x = xc[S::Q * l1 * C];
            if (!mul) return x;
            const float m = l1 < 8 ? sa[S::Q * l1 * C] : slab[(S::L - S::Q * l1 - l2) * C + ca];
            return make_float2(x.x * m, x.y * m);
          },
          [&](int m1) { return cconj(__ldg(twm + m1 * 32 + l2)); });
      __syncthreads();
      // the slab (and, after the last shell, the tile) has been read: fetch the next
      if (s + 1 < nshells) {
        if (mul) load_slab(s + 1, off);
      } else if (tn < ntiles) {
        stage(tn);
        if (mul) load_slab(0, off_next);
      }
      cp_async_commit();
      sreg_step_b<C, true>(T, cb, m1, hb, out + (int64_t)s * out_stride + i0 + cb, v.sl,
                           i0 + cb < v.inner ? rmask : 0u);
      cp_async_wait<0>();
      __syncthreads();
    }
    off = off_next;
  }
}

}  // namespace fft
}  // namespace ck
