// ck_xc16.cu -- the fused inverse-x + sums kernels for 9..16 shells.
#include "ck_xc_inst.cuh"

namespace ck {
namespace fft {

cudaError_t run_xc16(int M, const float2* spec, int64_t spec_stride, const float* w0, int nx, int px, int64_t rows,
                     int ny, const int* box, int nshells, const FftLen& f, const float2* stw, const float2* tw,
                     int max_ctas, int* ctas, double* partials, int* status, cudaStream_t st) {
  return run_xc_ns<16>(M, spec, spec_stride, w0, nx, px, rows, ny, box, nshells, f, stw, tw, max_ctas, ctas, partials,
                       status, st);
}

}  // namespace fft
}  // namespace ck
