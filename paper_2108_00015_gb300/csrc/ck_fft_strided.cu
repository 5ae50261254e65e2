// ck_fft_strided.cu -- instantiations of the strided-axis (y, z) FFT pass and
// of the multi-shell inverse z pass: 512-point axes run the register
// two-step kernels (ck_fft_sreg.cuh) unless the caller asks for row-ordered
// stores, the lengths of the grids in use (32 ... 512 cells per axis) the
// compile-time Stockham kernels, and any other length the runtime version.
//
// Row-ordered stores: the Stockham kernel's last iteration writes 8
// consecutive rows of the tile per warp instruction, the register kernel's
// step B rows 128 apart.  On the 16-shell inverse y pass (8.6 GB in place,
// rows 2 KB apart) the first sustained 5.2 TB/s on a GB300 and the second
// 4.0 TB/s, while on single-field passes the register kernel is faster.
#include <algorithm>

#include "ck_fft_core.cuh"
#include "ck_fft_sreg.cuh"

namespace ck {
namespace fft {

// Tile width of the register kernels (columns per tile, 32 threads per column).
constexpr int kSregC = 8;
constexpr int kZregC = 8;

template <int C>
static void run_sreg512(bool inv, const float2* in, float2* out, const StridedView& v, const float2* tw, int sm_count,
                        cudaStream_t st) {
  using S = Sreg<C>;
  const size_t sm = S::plain_bytes;
  const int64_t ntiles = v.n_outer * ((v.inner + C - 1) / C);
  auto go = [&](auto kernel) {
    allow_smem(kernel, sm);
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, S::NT, sm) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sm_count * occ));
    kernel<<<grid, S::NT, sm, st>>>(in, out, v, tw);
  };
  if (inv) go(sreg512_kernel<C, true>);
  else go(sreg512_kernel<C, false>);
}

template <int C>
static void run_zreg512(const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                        const float2* tw, const KhatArgs& K, int sm_count, cudaStream_t st) {
  using S = Sreg<C>;
  const size_t sm = S::multi_bytes;
  const int64_t ntiles = (v.inner + C - 1) / C;
  allow_smem(zreg512_kernel<C>, sm);
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, zreg512_kernel<C>, S::NT, sm) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sm_count * occ));
  zreg512_kernel<C><<<grid, S::NT, sm, st>>>(in, out, out_stride, nshells, v, tw, K);
}

template <int LC>
static void run_strided(bool inv, const float2* in, float2* out, const StridedView& v, const FftLen& f,
                        const float2* stw, int sm_count, cudaStream_t st) {
  const int L = LC > 0 ? LC : f.n;
  const size_t sm = strided_smem(L);
  const int64_t ntiles = v.n_outer * ((v.inner + kT - 1) / kT);
  if (inv) {
    allow_smem(strided_kernel<LC, true>, sm);
    strided_kernel<LC, true><<<persistent_grid(strided_kernel<LC, true>, sm, sm_count, ntiles), kThreads, sm, st>>>(
        in, out, v, f, stw);
  } else {
    allow_smem(strided_kernel<LC, false>, sm);
    strided_kernel<LC, false><<<persistent_grid(strided_kernel<LC, false>, sm, sm_count, ntiles), kThreads, sm, st>>>(
        in, out, v, f, stw);
  }
}

template <int LC>
static void run_zmulti(const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                       const FftLen& f, const float2* stw, const KhatArgs& K, int sm_count, cudaStream_t st) {
  const int L = LC > 0 ? LC : f.n;
  const size_t sm = zmulti_smem(L);
  const int64_t ntiles = (v.inner + kT - 1) / kT;
  allow_smem(zmulti_kernel<LC>, sm);
  zmulti_kernel<LC><<<persistent_grid(zmulti_kernel<LC>, sm, sm_count, ntiles), kThreads, sm, st>>>(
      in, out, out_stride, nshells, v, f, stw, K);
}

#define CK_LENGTHS(X) X(32) X(128) X(160) X(192) X(240) X(256) X(288) X(320) X(384) X(512)

void launch_strided(int L, bool inv, const float2* in, float2* out, const StridedView& v, const FftLen& f,
                    const float2* stw, const float2* tw, bool row_ordered, int sm_count, cudaStream_t st) {
  if (L == 512 && !row_ordered) {
    run_sreg512<kSregC>(inv, in, out, v, tw, sm_count, st);
    return;
  }
  switch (L) {
#define CK_CASE(N) case N: run_strided<N>(inv, in, out, v, f, stw, sm_count, st); return;
    CK_LENGTHS(CK_CASE)
#undef CK_CASE
    default: run_strided<0>(inv, in, out, v, f, stw, sm_count, st);
  }
}

void launch_zmulti(int L, const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                   const FftLen& f, const float2* stw, const float2* tw, const KhatArgs& K, int sm_count,
                   cudaStream_t st) {
  if (L == 512) {
    run_zreg512<kZregC>(in, out, out_stride, nshells, v, tw, K, sm_count, st);
    return;
  }
  switch (L) {
#define CK_CASE(N) case N: run_zmulti<N>(in, out, out_stride, nshells, v, f, stw, K, sm_count, st); return;
    CK_LENGTHS(CK_CASE)
#undef CK_CASE
    default: run_zmulti<0>(in, out, out_stride, nshells, v, f, stw, K, sm_count, st);
  }
}

}  // namespace fft
}  // namespace ck
