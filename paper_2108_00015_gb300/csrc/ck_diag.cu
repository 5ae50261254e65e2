// ck_diag.cu -- the equidistant n-point functions of Eq. 14:
// xi_n(s, .., s) = sum_r W0 W_s^(n-1) / sum_r B0 B_s^(n-1), for every shell s
// and orders 2..5, from one pass over the bank (O(N_c N_s) instead of every
// multiset).  The denominators are the (s, .., s) entries of the random
// field's raw sums the plan keeps, times alpha^n.
//  * diag_sums_kernel: CTA (s, b) sums W0 W_s^k, k = 1..4, over cells
//    b DG_CELLS .. + DG_CELLS - 1 (16-byte loads; a thread's FP32 sums over
//    its 32 cells flushed to FP64; the CTA's in a fixed tree).  The shell is
//    the fastest grid index, so the CTAs of one cell range run together and
//    read W0 from L2.
//  * diag_reduce_kernel: one warp per (k, s) sums the cell blocks (lanes
//    stride the blocks, then a fixed shuffle tree): the same result from run
//    to run.
//  * diag_finalize_kernel: num, den and xi for the requested orders; plans
//    with the fused order-2/3 pass (no bank) read the numerators from their
//    packed sums instead.
#include <algorithm>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {

namespace {

constexpr int DG_THREADS = 256;
constexpr int DG_CELLS = DG_THREADS * 32;  // cells per CTA: 32 per thread
constexpr int DG_K = CK_MAX_ORDER - 1;      // powers W_s^1 .. W_s^4

__global__ void __launch_bounds__(DG_THREADS) diag_sums_kernel(const float* __restrict__ w0,
                                                               const float* __restrict__ bank, int64_t bstride,
                                                               int64_t nc, int ns, double* __restrict__ partials) {
  __shared__ double red[DG_THREADS / 32][DG_K];
  const int s = blockIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * DG_CELLS;
  const int64_t c1 = std::min<int64_t>(nc, c0 + DG_CELLS);
  const float* ws = bank + (int64_t)s * bstride;
  float f[DG_K] = {0.f, 0.f, 0.f, 0.f};
  // 16-byte loads over whole groups of 4 cells (c0, w0, the bank rows and
  // bstride are multiples of 4 floats), the ragged end one cell at a time
  const int64_t c4 = c0 + (c1 - c0) / 4 * 4;
  for (int64_t c = c0 + 4 * (int64_t)threadIdx.x; c < c4; c += 4 * DG_THREADS) {
    const float4 a = *reinterpret_cast<const float4*>(w0 + c);
    const float4 w = *reinterpret_cast<const float4*>(ws + c);
    const float av[4] = {a.x, a.y, a.z, a.w}, wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float t = av[e] * wv[e];
#pragma unroll
      for (int k = 0; k < DG_K; ++k) {
        f[k] += t;
        t *= wv[e];
      }
    }
  }
  for (int64_t c = c4 + threadIdx.x; c < c1; c += DG_THREADS) {
    float t = w0[c] * ws[c];
#pragma unroll
    for (int k = 0; k < DG_K; ++k) {
      f[k] += t;
      t *= ws[c];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < DG_K; ++k) {
    double v = (double)f[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < DG_K) {
    double v = 0.0;
    for (int w = 0; w < DG_THREADS / 32; ++w) v += red[w][threadIdx.x];
    partials[((int64_t)blockIdx.y * ns + s) * DG_K + threadIdx.x] = v;
  }
}

// out[k][s] = sum over the cell blocks of the partials, k = 0..kmax - 1 (power k + 1)
__global__ void diag_reduce_kernel(const double* __restrict__ partials, int nblocks, int ns, int kmax,
                                   double* __restrict__ out) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)kmax * ns) return;
  const int k = (int)(t / ns), s = (int)(t % ns);
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += partials[((int64_t)b * ns + s) * DG_K + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) out[(int64_t)k * ns + s] = v;
}

struct DiagIndex {
  int64_t idx[CK_MAX_ORDER + 1][CK_MAX_SHELLS];  // packed multiset index of (s, .., s), order n
  int64_t dense_base[CK_MAX_ORDER + 1];          // outputs of order n in the dense area
};

// Order n, shell s: num from the diagonal sums (power n - 1) or, for fused
// plans, from the packed sums; den from the random field's raw sums.
__global__ void diag_finalize_kernel(const double* __restrict__ dsums, const double* __restrict__ packed,
                                     const double* __restrict__ den_raw, const DiagIndex di, int ns, int mask,
                                     DevState* st, double* __restrict__ dense, int64_t dense_total) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const double alpha = st->alpha;
  double an = alpha;
  for (int n = 2; n <= CK_MAX_ORDER; ++n) {
    an *= alpha;
    if (!((mask >> n) & 1)) continue;
    const int64_t r = di.idx[n][s];
    const double nu = packed ? packed[r] : dsums[(int64_t)(n - 2) * ns + s];
    const double de = den_raw[r] * an;
    double* xi = dense + di.dense_base[n] + s;
    xi[dense_total] = nu;
    xi[2 * dense_total] = de;
    if (de > 0.0) {
      *xi = nu / de;
    } else {
      *xi = __longlong_as_double(0x7ff8000000000000ll);
      set_status(&st->status, CK_ERR_ZERO_DENOM);
    }
  }
}

// (s, .., s) in packed multiset order (and the dense output offsets) per order
DiagIndex diag_index(const Plan& p) {
  DiagIndex di;
  int ms[CK_MAX_ORDER];
  for (int n = 0; n <= CK_MAX_ORDER; ++n) {
    di.dense_base[n] = p.dense_base[n];
    for (int s = 0; s < CK_MAX_SHELLS; ++s) {
      di.idx[n][s] = 0;
      if (n < 2 || n > p.max_order || s >= p.ns) continue;
      for (int i = 0; i < n - 1; ++i) ms[i] = s;
      di.idx[n][s] = p.multiset_base[n] + host_multiset_rank(ms, n - 1, p.ns);
    }
  }
  return di;
}

// den_raw[(s, .., s) of order n] = dsums[n - 2][s]
__global__ void diag_scatter_kernel(const double* __restrict__ dsums, const DiagIndex di, int ns, int max_order,
                                    double* __restrict__ packed) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  for (int n = 2; n <= max_order; ++n) packed[di.idx[n][s]] = dsums[(int64_t)(n - 2) * ns + s];
}

// The plan's field (already transformed) through the inverse passes into the
// bank, then sum_r field W_s^k for every shell, k = 1..max_order - 1, into
// out[k - 1][s] (max_order - 1 rows of ns doubles).
ck_status launch_diag_bank_sums(Plan& p, double* out, cudaStream_t st) {
  launch_fft_inverse(p, p.spec, 0, p.ns, p.tmp, p.bank, p.field_stride, st);
  const int64_t nblocks = (p.nc + DG_CELLS - 1) / DG_CELLS;
  if ((size_t)nblocks * p.ns * DG_K > p.partials_cap) return CK_ERR_OOM;
  {
    ProfScope ps(p, ST_CONTRACT, 4.0 * (double)(p.ns + 1) * (double)p.nc, st);
    diag_sums_kernel<<<dim3((unsigned)p.ns, (unsigned)nblocks), DG_THREADS, 0, st>>>(p.field, p.bank, p.field_stride,
                                                                                     p.nc, p.ns, p.partials);
  }
  const int kmax = p.max_order - 1;
  ProfScope ps2(p, ST_REDUCE, 8.0 * (double)nblocks * p.ns * DG_K, st);
  const int64_t threads = (int64_t)kmax * p.ns * 32;
  diag_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(p.partials, (int)nblocks, p.ns, kmax, out);
  return cuda_status(cudaGetLastError());
}

}  // namespace

ck_status launch_diagonal(Plan& p, int mask, cudaStream_t st) {
  const DiagIndex di = diag_index(p);
  const double* packed = nullptr;
  double* dsums = p.sums;  // [max_order - 1][ns] when the bank is kept (each order has >= ns multisets)
  if (p.fused) {
    // no bank: the fused pass computes every order-2/3 multiset, the diagonal
    // among them, over the box of occupied cells (W_0 = N vanishes elsewhere)
    launch_support_box(p, 0, st);
    const ck_status s = launch_convolve_contract(p, p.field, p.sums, st, p.support);
    if (s != CK_OK) return s;
    packed = p.sums;
  } else {
    const ck_status s = launch_diag_bank_sums(p, dsums, st);
    if (s != CK_OK) return s;
  }
  ProfScope ps3(p, ST_FINALIZE, 0.0, st);
  diag_finalize_kernel<<<(p.ns + 63) / 64, 64, 0, st>>>(dsums, packed, p.den_raw, di, p.ns, mask, p.dstate, p.dense,
                                                          p.dense_total);
  return cuda_status(cudaGetLastError());
}

ck_status launch_diagonal_randoms(Plan& p, bool* full, cudaStream_t st) {
  if (p.fused) {  // the fused pass gives every multiset of the plan's orders
    *full = true;
    launch_support_box(p, 1, st);
    return launch_convolve_contract(p, p.field, p.den_raw, st, p.support);
  }
  *full = false;
  const ck_status s = launch_diag_bank_sums(p, p.sums, st);
  if (s != CK_OK) return s;
  diag_scatter_kernel<<<(p.ns + 63) / 64, 64, 0, st>>>(p.sums, diag_index(p), p.ns, p.max_order, p.den_raw);
  return cuda_status(cudaGetLastError());
}

}  // namespace ck
