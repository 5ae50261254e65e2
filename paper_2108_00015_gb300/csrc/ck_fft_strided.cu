// ck_fft_strided.cu -- instantiations of the strided-axis (y, z) FFT pass and
// of the multi-shell inverse z pass for the transform lengths of the grids in
// use (32 ... 512 cells per axis); other lengths use the runtime version.
#include <algorithm>

#include "ck_fft_core.cuh"

namespace ck {
namespace fft {

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
                    const float2* stw, int sm_count, cudaStream_t st) {
  switch (L) {
#define CK_CASE(N) case N: run_strided<N>(inv, in, out, v, f, stw, sm_count, st); return;
    CK_LENGTHS(CK_CASE)
#undef CK_CASE
    default: run_strided<0>(inv, in, out, v, f, stw, sm_count, st);
  }
}

void launch_zmulti(int L, const float2* in, float2* out, int64_t out_stride, int nshells, const StridedView& v,
                   const FftLen& f, const float2* stw, const KhatArgs& K, int sm_count, cudaStream_t st) {
  switch (L) {
#define CK_CASE(N) case N: run_zmulti<N>(in, out, out_stride, nshells, v, f, stw, K, sm_count, st); return;
    CK_LENGTHS(CK_CASE)
#undef CK_CASE
    default: run_zmulti<0>(in, out, out_stride, nshells, v, f, stw, K, sm_count, st);
  }
}

}  // namespace fft
}  // namespace ck
