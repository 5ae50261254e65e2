// ck_fft_strided.cu -- instantiations of the strided-axis (y, z) FFT pass and
// of the multi-shell inverse z pass: 512-point axes run the register
// two-step kernels (ck_fft_sreg.cuh), the other lengths of the grids in use
// (32 ... 384 cells per axis) the compile-time Stockham kernels, and any
// other length the runtime version.
//
// Tile width of the 512-point register kernels: 8 columns (256 threads, two
// CTAs per SM; three for the K^ z pass) for single-field passes, 16 columns
// (512 threads, one CTA per SM) when the caller asks for wide tiles.  On the 16-shell in-place inverse
// y pass (8.6 GB) a GB300 sustained 5.6 TB/s with 16 columns, 5.2 TB/s with
// the Stockham kernel and 4.0 TB/s with 8 columns; on single-field passes
// 8 columns are the fastest.
#include <algorithm>

#include "ck_fft_core.cuh"
#include "ck_fft_sreg.cuh"

namespace ck {
namespace fft {

// Default tile width of the register kernels (columns per tile, 32 threads
// per column); a plan's autotuner may choose 16 per pass.
constexpr int kSregC = 8;
constexpr int kZregC = 8;

template <int C>
static void run_sreg512(bool inv, const float2* in, float2* out, const StridedView& v, const float2* tw, int sm_count,
                        cudaStream_t st, const int* box, int nz, int mode) {
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
    kernel<<<grid, S::NT, sm, st>>>(in, out, v, tw, box, nz, mode);
  };
  if (inv) go(sreg512_kernel<C, true>);
  else go(sreg512_kernel<C, false>);
}

template <int C>
static void run_zreg512(const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                        const float2* tw, const KhatArgs& K, int sm_count, cudaStream_t st, const int* box) {
  using S = Sreg<C>;
  const size_t sm = S::multi_bytes;
  const int64_t ntiles = (v.inner + C - 1) / C;
  allow_smem(zreg512_kernel<C>, sm);
  // three 8-column CTAs (3 x 74.2 KB) need the largest shared-memory carveout
  cudaFuncSetAttribute(zreg512_kernel<C>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, zreg512_kernel<C>, S::NT, sm) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sm_count * occ));
  zreg512_kernel<C><<<grid, S::NT, sm, st>>>(in, out, out_stride, nshells, v, tw, K, box);
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

#define CK_LENGTHS(X) X(32) X(128) X(160) X(192) X(240) X(256) X(288) X(320) X(384)

void launch_strided(int L, bool inv, const float2* in, float2* out, const StridedView& v, const FftLen& f,
                    const float2* stw, const float2* tw, int cols, int sm_count, cudaStream_t st, const int* box,
                    int nz, int mode) {
  if (L == 512) {
    if (cols == 16) run_sreg512<16>(inv, in, out, v, tw, sm_count, st, box, nz, mode);
    else run_sreg512<kSregC>(inv, in, out, v, tw, sm_count, st, box, nz, mode);
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
                   cudaStream_t st, const int* box, int cols) {
  if (L == 512) {
    if (cols == 16) run_zreg512<16>(in, out, out_stride, nshells, v, tw, K, sm_count, st, box);
    else run_zreg512<kZregC>(in, out, out_stride, nshells, v, tw, K, sm_count, st, box);
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
