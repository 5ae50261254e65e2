// ck_xc.cu -- convolution and summation of one field in one pass over the
// shell spectra (Sec. 2.4-2.5, Eqs. 9-11): the inverse z (with the K^_s
// multiply) and y passes as in ck_fft.cu, then the x pass fused with the
// order-2 and order-3 sums (ck_xc.cuh), so that the bank W_s is never
// written to global memory.  Used by plans with FP32 sums, at most 16 shells
// and orders up to 3; the others run the separate passes and contraction.
#include <algorithm>

#include "ck_xc_inst.cuh"

namespace ck {
namespace fft {

cudaError_t run_xc16(int M, const float2* spec, int64_t spec_stride, const float* w0, int nx, int px, int64_t rows,
                     int ny, const int* box, int nshells, const FftLen& f, const float2* stw, const float2* tw,
                     int max_ctas, int* ctas, double* partials, int* status, cudaStream_t st);

}  // namespace fft


int xc_pad_shells(int ns) {
  if (ns <= 2) return 2;
  if (ns <= 4) return 4;
  if (ns <= 8) return 8;
  if (ns <= 16) return 16;
  return 0;
}

size_t xc_smem_bytes(int M, int ns_pad) {
  switch (ns_pad) {
    case 2: return fft::xc_smem_ns<2>(M);
    case 4: return fft::xc_smem_ns<4>(M);
    case 8: return fft::xc_smem_ns<8>(M);
    default: return fft::xc_smem_ns<16>(M);
  }
}

// Per-CTA partials of the padded layout -> packed per-order sums of the
// plan's shells, summed over CTAs in a fixed order (one warp per output).
__global__ void reduce_xc_kernel(const double* __restrict__ partials, int ctas, int nout_pad, int ns_pad, int ns,
                                 int max_order, int64_t base2, int64_t base3, double* __restrict__ out) {
  const int n2 = ns, n3 = max_order >= 3 ? ns * (ns + 1) / 2 : 0;
  // one warp per output
  const int o = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (o >= n2 + n3) return;  // whole warps
  int src;
  int64_t dst;
  if (o < n2) {
    src = o;
    dst = base2 + o;
  } else {
    // (a, b), a <= b, in lexicographic order over ns shells
    int r = o - n2, a = 0;
    while (r >= ns - a) {
      r -= ns - a;
      ++a;
    }
    const int b = a + r;
    src = ns_pad + a * ns_pad - a * (a - 1) / 2 + (b - a);
    dst = base3 + (o - n2);
  }
  // a fixed order: lane l adds the CTAs l, l + 32, ... in turn, then the
  // lanes' sums combine in a fixed butterfly (the same sum on every run)
  double s = 0.0;
  for (int c = lane; c < ctas; c += 32) s += __ldg(partials + (int64_t)c * nout_pad + src);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if (lane == 0) out[dst] = s;
}

ck_status launch_convolve_contract(Plan& p, const float* w0, double* sums, cudaStream_t st, const int* box) {
  const int nx = p.grid.n[0], ny = p.grid.n[1], nz = p.grid.n[2];
  const int M = nx / 2;
  const int ns_pad = xc_pad_shells(p.ns);
  if (ns_pad == 0 || p.max_order > 3) return CK_ERR_UNSUPPORTED;
  const int nout_pad = ns_pad + ns_pad * (ns_pad + 1) / 2;
  const int64_t rows = (int64_t)ny * nz;
  // at most two resident CTAs per SM
  const int max_ctas = (int)std::min<size_t>((size_t)2 * p.sm_count, p.partials_cap / nout_pad);
  int ctas = 0;

  launch_inverse_zy(p, p.spec, 0, p.ns, p.tmp, st, box);
  cudaError_t e;
  {
    const double H = (double)nz * ny * (nx / 2 + 1);
    // bytes: every row, or the box's rows (a half-spectrum row per shell and its N cells)
    ProfScope ps(p, ST_X_C2R_CONTRACT, box ? 0.0 : p.ns * 8.0 * H + 4.0 * (double)p.nc,
                 p.ns * 8.0 * (nx / 2 + 1) + 4.0 * nx, 0.0, box, st);
    const FftLen& f = p.fx_half;
    if (ns_pad == 16)
      e = fft::run_xc16(M, p.tmp, p.spec_elems, w0, nx, p.px, rows, ny, box, p.ns, f, p.stw[0], p.tw[0], max_ctas, &ctas,
                        p.partials, &p.dstate->status, st);
    else if (ns_pad == 8)
      e = fft::run_xc_ns<8>(M, p.tmp, p.spec_elems, w0, nx, p.px, rows, ny, box, p.ns, f, p.stw[0], p.tw[0], max_ctas,
                            &ctas, p.partials, &p.dstate->status, st);
    else if (ns_pad == 4)
      e = fft::run_xc_ns<4>(M, p.tmp, p.spec_elems, w0, nx, p.px, rows, ny, box, p.ns, f, p.stw[0], p.tw[0], max_ctas,
                            &ctas, p.partials, &p.dstate->status, st);
    else
      e = fft::run_xc_ns<2>(M, p.tmp, p.spec_elems, w0, nx, p.px, rows, ny, box, p.ns, f, p.stw[0], p.tw[0], max_ctas,
                            &ctas, p.partials, &p.dstate->status, st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  ProfScope ps2(p, ST_REDUCE, 8.0 * (double)ctas * nout_pad, st);
  const int nkeep = p.ns + (p.max_order >= 3 ? p.ns * (p.ns + 1) / 2 : 0);
  reduce_xc_kernel<<<(nkeep + 3) / 4, 128, 0, st>>>(p.partials, ctas, nout_pad, ns_pad, p.ns, p.max_order,
                                                   p.multiset_base[2], p.multiset_base[3], sums);
  return cuda_status(cudaGetLastError());
}

}  // namespace ck
