// ck_xc_inst.cuh -- host launchers of the fused inverse-x + sums kernels for
// one padded shell count NS (instantiated per translation unit so that the
// kernels compile in parallel).  Power-of-two half-lengths 16..256 run the
// register transform (xcr_contract_kernel), the others the shared-memory
// Stockham one (xc_contract_kernel).
#pragma once

#include <algorithm>

#include "ck_xc.cuh"

namespace ck {
namespace fft {

inline int xc_ctas(int64_t ntiles, int max_ctas) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, max_ctas));
}

template <int MC, int NS>
cudaError_t run_xc(const float2* spec, int64_t spec_stride, const float* w0, int nx, int px, int64_t rows, int ny,
                   const int* box, int nshells, const FftLen& f, const float2* stw, const float2* tw, int max_ctas,
                   int* ctas, double* partials, cudaStream_t st) {
  const int M = MC > 0 ? MC : nx / 2;
  const size_t sm = xc_layout(M, NS, MC > 0 ? tw_table_len(rplan(MC)) : xc_ntw(M)).total;
  *ctas = xc_ctas((rows + xc_rows(NS) - 1) / xc_rows(NS), max_ctas);
  cudaError_t e = cudaFuncSetAttribute(xc_contract_kernel<MC, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  xc_contract_kernel<MC, NS><<<*ctas, kThreads, sm, st>>>(spec, spec_stride, w0, nx, px, rows, ny, box, nshells, f,
                                                         stw, tw, partials);
  return cudaGetLastError();
}

template <int P, int Q, int NS>
cudaError_t run_xcr(const float2* spec, int64_t spec_stride, const float* w0, int px, int64_t rows, int ny,
                    const int* box, int nshells, const float2* tw, int max_ctas, int* ctas, double* partials,
                    int* status, cudaStream_t st) {
  using S = XcrShape<P, Q, NS>;
  if (px != S::LP) return cudaErrorInvalidValue;  // whole padded rows are staged
  *ctas = xc_ctas((rows + S::ROWS - 1) / S::ROWS, max_ctas);
  cudaError_t e = cudaFuncSetAttribute(xcr_contract_kernel<P, Q, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)S::total);
  if (e != cudaSuccess) return e;
  xcr_contract_kernel<P, Q, NS><<<*ctas, kThreads, S::total, st>>>(spec, spec_stride, w0, px, rows, ny, box, nshells,
                                                                   tw, partials, status);
  return cudaGetLastError();
}

#define CK_XC_LENGTHS(X) X(80) X(96) X(120) X(144) X(160) X(192)

template <int NS>
cudaError_t run_xc_ns(int M, const float2* spec, int64_t spec_stride, const float* w0, int nx, int px, int64_t rows,
                      int ny, const int* box, int nshells, const FftLen& f, const float2* stw, const float2* tw,
                      int max_ctas, int* ctas, double* partials, int* status, cudaStream_t st) {
  switch (M) {
    case 256: return run_xcr<16, 16, NS>(spec, spec_stride, w0, px, rows, ny, box, nshells, tw, max_ctas, ctas, partials,
                                       status, st);
    case 128: return run_xcr<16, 8, NS>(spec, spec_stride, w0, px, rows, ny, box, nshells, tw, max_ctas, ctas, partials,
                                       status, st);
    case 64: return run_xcr<8, 8, NS>(spec, spec_stride, w0, px, rows, ny, box, nshells, tw, max_ctas, ctas, partials,
                                       status, st);
    case 32: return run_xcr<8, 4, NS>(spec, spec_stride, w0, px, rows, ny, box, nshells, tw, max_ctas, ctas, partials,
                                       status, st);
    case 16: return run_xcr<4, 4, NS>(spec, spec_stride, w0, px, rows, ny, box, nshells, tw, max_ctas, ctas, partials,
                                       status, st);
#define CK_CASE(N)                                                                                              \
  case N:                                                                                                       \
    return run_xc<N, NS>(spec, spec_stride, w0, nx, px, rows, ny, box, nshells, f, stw, tw, max_ctas, ctas, partials, \
                         st);
    CK_XC_LENGTHS(CK_CASE)
#undef CK_CASE
    default:
      return run_xc<0, NS>(spec, spec_stride, w0, nx, px, rows, ny, box, nshells, f, stw, tw, max_ctas, ctas, partials,
                           st);
  }
}

// Shared memory of the fused pass for half-length M and padded shell count NS.
template <int NS>
size_t xc_smem_ns(int M) {
  switch (M) {
    case 256: return XcrShape<16, 16, NS>::total;
    case 128: return XcrShape<16, 8, NS>::total;
    case 64: return XcrShape<8, 8, NS>::total;
    case 32: return XcrShape<8, 4, NS>::total;
    case 16: return XcrShape<4, 4, NS>::total;
    default: return xc_layout(M, NS, xc_ntw(M)).total;
  }
}

}  // namespace fft
}  // namespace ck
