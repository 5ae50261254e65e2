// ck_fft_x.cu -- instantiations of the real x-axis FFT passes (half-length
// complex transform of M = n[0]/2 points) for the grid widths in use; other
// widths use the runtime version.
#include <algorithm>

#include "ck_fft_core.cuh"

namespace ck {
namespace fft {

template <int MC>
static void run_r2c(const float* in, float2* out, int nx, int px, int64_t rows, const FftLen& f, const float2* stw,
                    const float2* tw, int sm_count, cudaStream_t st, const int* box, int ny) {
  const size_t sm = xpass_smem(nx);
  const int64_t ntiles = (rows + kT - 1) / kT;
  allow_smem(x_r2c_kernel<MC>, sm);
  x_r2c_kernel<MC><<<persistent_grid(x_r2c_kernel<MC>, sm, sm_count, ntiles), kThreads, sm, st>>>(
      in, out, nx, px, rows, f, stw, tw, box, ny);
}

template <int MC>
static void run_c2r(const float2* in, float* out, int nx, int px, int64_t rows, int64_t rps, int64_t oss,
                    const FftLen& f, const float2* stw, const float2* tw, int sm_count, cudaStream_t st,
                    const int* box, int ny) {
  const size_t sm = xpass_smem(nx);
  const int64_t ntiles = (rows + kT - 1) / kT;  // the grid covers every row; a box visits fewer
  allow_smem(x_c2r_kernel<MC>, sm);
  x_c2r_kernel<MC><<<persistent_grid(x_c2r_kernel<MC>, sm, sm_count, ntiles), kThreads, sm, st>>>(
      in, out, nx, px, rows, rps, oss, f, stw, tw, box, ny);
}

#define CK_HALF_LENGTHS(X) X(16) X(64) X(80) X(96) X(120) X(128) X(144) X(160) X(192) X(256)

void launch_x_r2c(int M, const float* in, float2* out, int nx, int px, int64_t rows, const FftLen& f,
                  const float2* stw, const float2* tw, int sm_count, cudaStream_t st, const int* box, int ny) {
  // 512-cell rows: the register form (ck_fft_xr.cu)
  if (M == 256) {
    launch_xr2c_reg(in, out, px, rows, tw, sm_count, st, box, ny);
    return;
  }
  switch (M) {
#define CK_CASE(N) case N: run_r2c<N>(in, out, nx, px, rows, f, stw, tw, sm_count, st, box, ny); return;
    CK_HALF_LENGTHS(CK_CASE)
#undef CK_CASE
    default: run_r2c<0>(in, out, nx, px, rows, f, stw, tw, sm_count, st, box, ny);
  }
}

void launch_x_c2r(int M, const float2* in, float* out, int nx, int px, int64_t rows, int64_t rows_per_shell,
                  int64_t out_shell_stride, const FftLen& f, const float2* stw, const float2* tw, int sm_count,
                  cudaStream_t st, const int* box, int ny) {
  // 512-cell rows (pitch 260): the register form (ck_fft_xr.cu)
  if (M == 256 && px == M + 4) {
    launch_xc2r_reg(in, out, px, rows, rows_per_shell, out_shell_stride, tw, sm_count, st, box, ny);
    return;
  }
  switch (M) {
#define CK_CASE(N)                                                                                            \
  case N:                                                                                                     \
    run_c2r<N>(in, out, nx, px, rows, rows_per_shell, out_shell_stride, f, stw, tw, sm_count, st, box, ny); \
    return;
    CK_HALF_LENGTHS(CK_CASE)
#undef CK_CASE
    default: run_c2r<0>(in, out, nx, px, rows, rows_per_shell, out_shell_stride, f, stw, tw, sm_count, st, box, ny);
  }
}

}  // namespace fft
}  // namespace ck
