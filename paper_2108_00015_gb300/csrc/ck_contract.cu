// ck_contract.cu -- the summation stage (Sec. 2.5, Eqs. 11-14): for every
// multiset s_1 <= .. <= s_{n-1}, sum_r W0(r) prod_i W_{s_i}(r), n = 2..5,
// with a fixed-order FP64 reduction across blocks, then xi_n = num / den.
//
// Two kernels:
//  * contract_reg: few outputs (N_s <= 16 and n <= 3, or N_s <= 5 and
//    n <= 5).  One warp streams cell chunks of W0 and every W_s into a
//    six-stage shared-memory ring with bulk asynchronous copies of 1792 bytes
//    (mbarrier completion); seven consumer warps take two cells per thread
//    and chunk and keep every product sum in registers (FP32 over 64 chunks,
//    then warp-reduced into FP64 in shared memory).  HBM-bound: it reads each
//    W_s once.
//  * the blocked product below on the fifth-generation tensor cores with
//    split-TF32 operands (ck_umma.cu) for CK_PREC_SPLIT_TF32 plans that keep
//    the bank (n >= 4 or more than 16 shells).
//  * contract_blocked: the general case as a blocked product
//    T[p][q] = sum_r A_p(r) B_q(r) with A_p = W0 W_i W_j and B_q = W_k W_l
//    generated per cell chunk in shared memory (64 x 64 output tiles, 4 x 4
//    per thread).  Only tiles holding a canonical (p, q) are launched:
//    n=2: A=W0, B=W_c;  n=3: A=W0 W_a, B=W_c, a <= c;  n=4: A=W0 W_a W_b,
//    B=W_c, b <= c;  n=5: A=W0 W_a W_b, B=W_c W_d, b <= c.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ck_device.cuh"
#include "ck_internal.h"
#include "ck_sums.cuh"

namespace ck {

constexpr int RK_CW = 7;                 // consumer warps
constexpr int RK_CPT = 2;                // cells per consumer thread and chunk
constexpr int RK_KC = 32 * RK_CW * RK_CPT;  // cells per chunk (1792-byte copies)
constexpr int RK_STAGES = 6;             // ring depth
constexpr int RK_FLUSH = 64;             // chunks between FP32 -> FP64 flushes

// Orders 2 and 3 for the shells a in [A0, A1) only, in the local order
// (a, then b >= a): acc[i] for n = 2 at (a), then n = 3 at (a, a..NS-1).
template <int NS, int A0, int A1>
__device__ __forceinline__ void reg_accumulate_range(float* acc, const float* v) {
  int i = 0;
#pragma unroll
  for (int a = A0; a < A1; ++a) {
    const float p1 = v[0] * v[1 + a];
    acc[i++] += p1;
#pragma unroll
    for (int b = a; b < NS; ++b) acc[i++] += p1 * v[1 + b];
  }
}

__host__ __device__ constexpr int rank3(int ns, int a, int b) {  // (a <= b) in lexicographic order
  return a * ns - a * (a - 1) / 2 + (b - a);
}

// Flush the local accumulators of shells [A0, A1) into the warp's FP64 row
// (global order: n = 2 at a, n = 3 at ns + rank3(a, b)).
template <int NS, int A0, int A1>
__device__ __forceinline__ void reg_flush_range(float* acc, double* wacc, int lane) {
  int i = 0;
#pragma unroll
  for (int a = A0; a < A1; ++a) {
#pragma unroll
    for (int b = a - 1; b < NS; ++b) {
      float t = acc[i];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
      const int o = b < a ? a : NS + rank3(NS, a, b);
      if (lane == 0) wacc[o] += (double)t;
      acc[i++] = 0.0f;
    }
  }
}

// Split of the shells between two consumer groups with about half of the
// order-2 and order-3 outputs each.
__host__ __device__ constexpr int split_shell(int ns) {
  const int total = ns + ns * (ns + 1) / 2;
  int acc = 0;
  for (int a = 0; a < ns; ++a) {
    acc += 1 + (ns - a);
    if (2 * acc >= total) return a + 1;
  }
  return ns;
}

__host__ __device__ constexpr int outs_range(int ns, int a0, int a1) {
  int t = 0;
  for (int a = a0; a < a1; ++a) t += 1 + (ns - a);
  return t;
}

// Test of the timeout path (ck_debug_force_timeout): when nonzero, every
// consumer warp of contract_reg_kernel first waits, with this limit in ns,
// on an mbarrier that nothing arrives at, so it gives up, records
// CK_ERR_TIMEOUT and consumes nothing; the producer's waits and its drain of
// the copies in flight keep the default limit.
__device__ uint64_t g_force_timeout_ns = 0;

// G = 1: every consumer thread keeps all outputs.  G = 2 (orders <= 3 only):
// two groups of RK_CW consumer warps see every cell, each keeping the sums of
// half of the shells, so twice as many warps fit with half the registers.
template <int NS, int MAXN, int G>
__global__ void __launch_bounds__(32 * (RK_CW * G + 1), 1)
    contract_reg_kernel(const float* __restrict__ w0, const float* __restrict__ bank, int64_t bstride, int64_t nc,
                        const int* __restrict__ box, int64_t plane, double* __restrict__ partials, int* status) {
  static_assert(G == 1 || (G == 2 && MAXN == 3), "two consumer groups only for orders <= 3");
  constexpr int NARR = NS + 1;
  constexpr int NOUT = RegOut<NS, MAXN>::total;
  constexpr int CWT = RK_CW * G;
  constexpr int SPLIT = split_shell(NS);
  constexpr int GOUT0 = outs_range(NS, 0, SPLIT), GOUT1 = outs_range(NS, SPLIT, NS);
  constexpr int NACC = G == 1 ? NOUT : (GOUT0 > GOUT1 ? GOUT0 : GOUT1);
  extern __shared__ __align__(128) unsigned char smem[];
  float* buf = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)RK_STAGES * NARR * RK_KC * 4);
  uint64_t* empty = full + RK_STAGES;
  int* consumed_min = reinterpret_cast<int*>(empty + RK_STAGES);
  uint64_t* never = empty + RK_STAGES + 1;  // armed by nobody (ck_debug_force_timeout)
  double* wacc = reinterpret_cast<double*>(empty + RK_STAGES + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // chunks of the visited cells [cr.lo, cr.hi), shared out evenly over the CTAs
  const CellRange cr = box_cells(box, plane, nc);
  const int64_t nchunks = (cr.hi - cr.lo + RK_KC - 1) / RK_KC;
  const int64_t chunks_per_cta = (nchunks + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = (int64_t)blockIdx.x * chunks_per_cta;
  const int64_t c1 = std::min<int64_t>(c0 + chunks_per_cta, nchunks);
  const int nit = (int)std::max<int64_t>(c1 - c0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < RK_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CWT);
    }
    mbar_init(never, 1);
    *consumed_min = nit;
    fence_async_shared();
  }
  for (int i = threadIdx.x; i < CWT * NOUT; i += blockDim.x) wacc[i] = 0.0;
  __syncthreads();
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nit; ++it) {
        const int st = it % RK_STAGES;
        const uint32_t ph = (uint32_t)(it / RK_STAGES) & 1u;
        if (it >= RK_STAGES && !mbar_wait(&empty[st], ph ^ 1u, status)) break;
        const int64_t cell0 = cr.lo + (c0 + it) * RK_KC;
        const int64_t rem = std::min<int64_t>(RK_KC, cr.hi - cell0);
        const uint32_t bytes = (uint32_t)((rem / 4) * 16);
        mbar_arrive_expect_tx(&full[st], bytes * NARR);
        if (bytes) {
          float* dst = buf + (size_t)st * NARR * RK_KC;
          bulk_g2s(dst, w0 + cell0, bytes, &full[st]);
#pragma unroll 1
          for (int a = 1; a < NARR; ++a) bulk_g2s(dst + a * RK_KC, bank + (a - 1) * bstride + cell0, bytes, &full[st]);
        }
        issued = it + 1;
      }
    }
  } else {
    const int grp = (warp - 1) / RK_CW;
    const int ct = threadIdx.x - 32 - grp * 32 * RK_CW;
    double* wrow = wacc + (warp - 1) * NOUT;
    float acc[NACC];
#pragma unroll
    for (int o = 0; o < NACC; ++o) acc[o] = 0.0f;
    int since = 0, done = 0;
    const uint64_t forced = g_force_timeout_ns;
    const int nrun = forced != 0 && !mbar_wait_for(never, 0u, status, forced) ? 0 : nit;
    for (int it = 0; it < nrun; ++it) {
      const int st = it % RK_STAGES;
      const uint32_t ph = (uint32_t)(it / RK_STAGES) & 1u;
      if (!mbar_wait(&full[st], ph, status)) break;
      const int64_t cell0 = cr.lo + (c0 + it) * RK_KC;
      const int64_t rem = std::min<int64_t>(RK_KC, cr.hi - cell0);
      const int64_t whole = rem / 4 * 4;
#pragma unroll
      for (int u = 0; u < RK_CPT; ++u) {
        const int cc = u * 32 * RK_CW + ct;
        if (cc < rem) {
          float v[NARR];
          if (cc < whole) {
            const float* src = buf + (size_t)st * NARR * RK_KC + cc;
#pragma unroll
            for (int a = 0; a < NARR; ++a) v[a] = src[a * RK_KC];
          } else {
            v[0] = __ldg(w0 + cell0 + cc);
#pragma unroll
            for (int a = 1; a < NARR; ++a) v[a] = __ldg(bank + (a - 1) * bstride + cell0 + cc);
          }
          if constexpr (G == 1) reg_accumulate<NS, MAXN>(acc, v);
          else if (grp == 0) reg_accumulate_range<NS, 0, SPLIT>(acc, v);
          else reg_accumulate_range<NS, SPLIT, NS>(acc, v);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      done = it + 1;
      if (++since == RK_FLUSH) {
        if constexpr (G == 1) reg_flush<NOUT>(acc, wrow, lane);
        else if (grp == 0) reg_flush_range<NS, 0, SPLIT>(acc, wrow, lane);
        else reg_flush_range<NS, SPLIT, NS>(acc, wrow, lane);
        since = 0;
      }
    }
    if constexpr (G == 1) reg_flush<NOUT>(acc, wrow, lane);
    else if (grp == 0) reg_flush_range<NS, 0, SPLIT>(acc, wrow, lane);
    else reg_flush_range<NS, SPLIT, NS>(acc, wrow, lane);
    if (lane == 0) atomicMin(consumed_min, done);
  }
  __syncthreads();
  // After a timeout, wait (bounded) for copies that were issued but not consumed.
  if (warp == 0 && lane == 0) {
    for (int it = *consumed_min; it < issued; ++it)
      if (!mbar_wait(&full[it % RK_STAGES], (uint32_t)(it / RK_STAGES) & 1u, status)) break;
  }
  for (int o = threadIdx.x; o < NOUT; o += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < CWT; ++w) s += wacc[w * NOUT + o];
    partials[(int64_t)blockIdx.x * NOUT + o] = s;
  }
}

// two consumer groups for the larger order-3 shell counts
template <int NS, int MAXN>
constexpr int reg_groups() { return 1; }  // two groups measured slower (shared-memory reads double)

template <int NS, int MAXN>
static size_t reg_smem() {
  return (size_t)RK_STAGES * (NS + 1) * RK_KC * 4 + (2 * RK_STAGES + 2) * 8 +
         (size_t)RK_CW * reg_groups<NS, MAXN>() * RegOut<NS, MAXN>::total * 8;
}

template <int NS, int MAXN>
static cudaError_t launch_reg_t(const float* w0, const float* bank, int64_t bstride, int64_t nc, int ctas,
                                const int* box, int64_t plane, double* partials, int* status, cudaStream_t st) {
  constexpr int G = reg_groups<NS, MAXN>();
  const size_t sm = reg_smem<NS, MAXN>();
  cudaError_t e = cudaFuncSetAttribute(contract_reg_kernel<NS, MAXN, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  contract_reg_kernel<NS, MAXN, G><<<ctas, 32 * (RK_CW * G + 1), sm, st>>>(w0, bank, bstride, nc, box, plane, partials,
                                                                           status);
  return cudaGetLastError();
}

static int reg_nout(int ns, int maxn) {
  int t = ns;
  if (maxn >= 3) t += cmb(ns + 1, 2);
  if (maxn >= 4) t += cmb(ns + 2, 3);
  if (maxn >= 5) t += cmb(ns + 3, 4);
  return t;
}

#define CK_REG_CASE3(N) \
  case N: return launch_reg_t<N, 3>(w0, bank, bstride, nc, ctas, box, plane, partials, status, st);
#define CK_REG_CASE5(N) \
  case N: return launch_reg_t<N, 5>(w0, bank, bstride, nc, ctas, box, plane, partials, status, st);

static cudaError_t launch_reg(int ns, int maxn, const float* w0, const float* bank, int64_t bstride, int64_t nc,
                              int ctas, const int* box, int64_t plane, double* partials, int* status,
                              cudaStream_t st) {
  if (maxn <= 3) {
    switch (ns) {
      CK_REG_CASE3(1) CK_REG_CASE3(2) CK_REG_CASE3(3) CK_REG_CASE3(4) CK_REG_CASE3(5) CK_REG_CASE3(6)
      CK_REG_CASE3(7) CK_REG_CASE3(8) CK_REG_CASE3(9) CK_REG_CASE3(10) CK_REG_CASE3(11) CK_REG_CASE3(12)
      CK_REG_CASE3(13) CK_REG_CASE3(14) CK_REG_CASE3(15) CK_REG_CASE3(16)
      default: break;
    }
  } else {
    switch (ns) {
      CK_REG_CASE5(1) CK_REG_CASE5(2) CK_REG_CASE5(3) CK_REG_CASE5(4) CK_REG_CASE5(5)
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

// Sum the register kernel's per-CTA partials in CTA order into the packed
// per-order layout (orders beyond the plan's max_order are dropped).
__global__ void reduce_reg_kernel(const double* __restrict__ partials, int ctas, int nout, int nkeep,
                                  double* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nkeep) return;
  double s = 0.0;
  for (int c = 0; c < ctas; ++c) s += partials[(int64_t)c * nout + o];
  out[o] = s;
}

// ---------------------------------------------------------------------------
// blocked kernel

constexpr int BK_T = 64;   // output tile side
constexpr int BK_FLUSH = 32;
// cells per chunk: 32 for FP32 operands, 16 for FP64 (static shared memory < 48 KB)
template <typename T>
constexpr int bk_kc() { return sizeof(T) == 4 ? 32 : 16; }

template <typename T>
__global__ void __launch_bounds__(256) contract_blocked_kernel(const float* __restrict__ w0, const float* __restrict__ bank,
                                                               int64_t bstride, int64_t nc, int ns,
                                                               const int2* __restrict__ rowdesc, int rows,
                                                               const int2* __restrict__ coldesc, int cols,
                                                               const int2* __restrict__ tiles, int ntiles,
                                                               const int* __restrict__ box, int64_t plane,
                                                               double* __restrict__ partials) {
  constexpr int BK_KC = bk_kc<T>();
  __shared__ T ws[CK_MAX_SHELLS + 1][BK_KC];
  __shared__ __align__(16) T As[BK_KC][BK_T];
  __shared__ __align__(16) T Bs[BK_KC][BK_T];
  __shared__ int2 rd[BK_T], cd[BK_T];
  const int tid = threadIdx.x;
  const int2 tile = tiles[blockIdx.x];
  if (tid < BK_T) {
    const int p = tile.x + tid;
    rd[tid] = p < rows ? rowdesc[p] : make_int2(-2, -2);
  } else if (tid < 2 * BK_T) {
    const int q = tile.y + tid - BK_T;
    cd[tid - BK_T] = q < cols ? coldesc[q] : make_int2(-2, -2);
  }
  const int ty = tid / 16, tx = tid % 16;
  T acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = T(0); dacc[i][j] = 0.0; }
  int64_t beg, end;  // this split's part of the visited cells (32-cell multiples)
  split_cells(box_cells(box, plane, nc), gridDim.y, 32, blockIdx.y, &beg, &end);
  int since = 0;
  __syncthreads();
  for (int64_t c0 = beg; c0 < end; c0 += BK_KC) {
    for (int idx = tid; idx < (ns + 1) * BK_KC; idx += 256) {
      const int a = idx / BK_KC, k = idx - a * BK_KC;
      const int64_t cell = c0 + k;
      float v = 0.0f;
      if (cell < end) v = a == 0 ? __ldg(w0 + cell) : __ldg(bank + (int64_t)(a - 1) * bstride + cell);
      ws[a][k] = (T)v;
    }
    __syncthreads();
    for (int idx = tid; idx < BK_KC * BK_T; idx += 256) {
      const int k = idx / BK_T, p = idx - k * BK_T;
      const int2 d = rd[p];
      T va = T(0);
      if (d.x != -2) {
        va = ws[0][k];
        if (d.x >= 0) va *= ws[1 + d.x][k];
        if (d.y >= 0) va *= ws[1 + d.y][k];
      }
      As[k][p] = va;
      const int2 e = cd[p];
      T vb = T(0);
      if (e.x != -2) {
        vb = T(1);
        if (e.x >= 0) vb *= ws[1 + e.x][k];
        if (e.y >= 0) vb *= ws[1 + e.y][k];
      }
      Bs[k][p] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < BK_KC; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[k][ty * 4 + i]; b[i] = Bs[k][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
    if (++since == BK_FLUSH) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { dacc[i][j] += (double)acc[i][j]; acc[i][j] = T(0); }
      since = 0;
    }
  }
  double* out = partials + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (BK_T * BK_T);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * BK_T + tx * 4 + j] = dacc[i][j] + (double)acc[i][j];
}

// Rank of a sorted multiset s[0..k) over ns symbols in lexicographic order.
__host__ __device__ inline int64_t multiset_rank(const int* s, int k, int ns) {
  int64_t r = 0;
  int prev = 0;
  for (int t = 0; t < k; ++t) {
    for (int v = prev; v < s[t]; ++v) {
      // multisets of size k-t-1 over symbols [v, ns)
      const int n = ns - v + (k - t - 1) - 1, kk = k - t - 1;
      int64_t c = 1;
      for (int i = 1; i <= kk; ++i) c = c * (n - kk + i) / i;
      r += c;
    }
    prev = s[t];
  }
  return r;
}

// Which order (and multiset) a (row, column) pair of the blocked product
// computes, or 0 if it is not the canonical pair of a requested order.
__host__ __device__ inline int canonical(int2 rd, int2 cd, int mask, int* ms) {
  if (rd.x == -2 || cd.x == -2) return 0;
  const int dA = (rd.x >= 0) + (rd.y >= 0);
  const int dB = (cd.x >= 0) + (cd.y >= 0);
  int n = 0;
  if (dA == 0 && dB == 1) n = 2;
  else if (dA == 1 && dB == 1 && rd.x <= cd.x) n = 3;
  else if (dA == 2 && dB == 1 && rd.y <= cd.x) n = 4;
  else if (dA == 2 && dB == 2 && rd.y <= cd.x) n = 5;
  if (n == 0 || !((mask >> n) & 1)) return 0;
  int k = 0;
  if (rd.x >= 0) ms[k++] = rd.x;
  if (rd.y >= 0) ms[k++] = rd.y;
  if (cd.x >= 0) ms[k++] = cd.x;
  if (cd.y >= 0) ms[k++] = cd.y;
  return n;
}

struct OrderBases {
  int64_t base[CK_MAX_ORDER + 1];
};

__global__ void reduce_blocked_kernel(const double* __restrict__ partials, int splits, int ntiles,
                                      const int2* __restrict__ tiles, const int2* __restrict__ rowdesc, int rows,
                                      const int2* __restrict__ coldesc, int cols, int mask, int ns, OrderBases B,
                                      double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ntiles * BK_T * BK_T) return;
  const int tile = (int)(t / (BK_T * BK_T));
  const int pq = (int)(t - (int64_t)tile * BK_T * BK_T);
  const int p = tiles[tile].x + pq / BK_T, q = tiles[tile].y + pq % BK_T;
  if (p >= rows || q >= cols) return;
  int ms[4];
  const int n = canonical(rowdesc[p], coldesc[q], mask, ms);
  if (!n) return;
  double s = 0.0;
  for (int sp = 0; sp < splits; ++sp) s += partials[((int64_t)sp * ntiles + tile) * (BK_T * BK_T) + pq];
  out[B.base[n] + multiset_rank(ms, n - 1, ns)] = s;
}

// ---------------------------------------------------------------------------
// host: per-mask contraction plans

static int max_order_in(int mask) {
  int m = 0;
  for (int n = 2; n <= CK_MAX_ORDER; ++n)
    if ((mask >> n) & 1) m = n;
  return m;
}

ck_status contract_prepare(Plan& p, int mask) {
  if (p.cplan_ready[mask]) return CK_OK;
  ContractPlan& c = p.cplan[mask];
  c = ContractPlan();
  c.order_mask = mask;
  const int maxn = max_order_in(mask);
  const int ns = p.ns;
  // register kernel: plain FP32 plans with few outputs
  if (p.precision == CK_PREC_FP32 && ((ns <= 16 && maxn <= 3) || (ns <= 5 && maxn <= 5))) {
    c.use_reg = true;
    c.reg_maxn = maxn <= 3 ? 3 : 5;
    c.n_out_reg = reg_nout(ns, c.reg_maxn);
    c.ctas = p.sm_count;
    const int64_t nchunks = (p.nc + RK_KC - 1) / RK_KC;
    c.chunks_per_cta = (nchunks + c.ctas - 1) / c.ctas;
    c.partial_doubles = (size_t)c.ctas * c.n_out_reg;
    if (c.partial_doubles > p.partials_cap) return CK_ERR_OOM;
    p.cplan_ready[mask] = true;
    return CK_OK;
  }
  // blocked kernel operand descriptors
  std::vector<int2> rows, cols;
  if ((mask >> 2) & 1) rows.push_back(make_int2(-1, -1));
  if ((mask >> 3) & 1)
    for (int a = 0; a < ns; ++a) rows.push_back(make_int2(a, -1));
  if (((mask >> 4) & 1) || ((mask >> 5) & 1))
    for (int b = 0; b < ns; ++b)
      for (int a = 0; a <= b; ++a) rows.push_back(make_int2(a, b));  // sorted by (b, a)
  if (((mask >> 2) & 1) || ((mask >> 3) & 1) || ((mask >> 4) & 1))
    for (int k = 0; k < ns; ++k) cols.push_back(make_int2(k, -1));
  if ((mask >> 5) & 1)
    for (int k = 0; k < ns; ++k)
      for (int l = k; l < ns; ++l) cols.push_back(make_int2(k, l));  // sorted by (k, l)
  c.use_tc = p.precision == CK_PREC_SPLIT_TF32 || p.precision == CK_PREC_SPLIT_BF16 ||
             p.precision == CK_PREC_SPLIT_FP16;
  c.um_kind = p.precision == CK_PREC_SPLIT_BF16 ? 1 : (p.precision == CK_PREC_SPLIT_FP16 ? 2 : 0);
  c.rows = (int)rows.size();
  c.cols = (int)cols.size();
  const size_t slot = p.table_arena_cap / (1 << (CK_MAX_ORDER + 1));
  int2* base = reinterpret_cast<int2*>(p.table_arena + slot * mask);
  int ms[4];
  if (c.use_tc) {
    // tensor cores: per 128-row tile, the list of columns holding a
    // canonical (p, q) with one of its rows, cut into tiles of at most 256
    // columns; MMA N = the list length rounded up to 32
    std::vector<int4> tl;
    std::vector<int> clist;
    const int TM = umma_tile_rows();
    int tnmax = 0;
    for (int m0 = 0; m0 < (int)rows.size(); m0 += TM) {
      std::vector<int> need;
      for (int qq = 0; qq < (int)cols.size(); ++qq) {
        bool any = false;
        for (int pp = m0; pp < std::min<int>(m0 + TM, (int)rows.size()) && !any; ++pp)
          any = canonical(rows[pp], cols[qq], mask, ms) != 0;
        if (any) need.push_back(qq);
      }
      for (size_t i = 0; i < need.size(); i += 256) {
        const int cnt = (int)std::min<size_t>(256, need.size() - i);
        const int tn = (cnt + 31) / 32 * 32;
        tl.push_back(make_int4(m0, (int)clist.size(), tn, cnt));
        clist.insert(clist.end(), need.begin() + i, need.begin() + i + cnt);
      }
    }
    // thin tiles (few outputs) go last, to the CUDA cores: per MMA a thin
    // tile costs the tensor cores as much as a full one
    auto thin = [&](const int4& t) {
      const int live = std::min<int>(TM, (int)rows.size() - t.x);
      return t.w <= kThinMaxCols && live * t.w <= kThinMaxOut && umma_thin_smem(ns, live) <= (size_t)227 * 1024;
    };
    std::stable_partition(tl.begin(), tl.end(), [&](const int4& t) { return !thin(t); });
    c.um_ntc = 0;
    c.um_thin_rmax = 0;
    for (int4& t : tl)
      if (!thin(t)) {
        ++c.um_ntc;
        // narrow tiles: hi and lo of B side by side, two MMAs per k-step
        const int half = (t.w + 15) / 16 * 16;
        if (t.w <= p.tune.tc_stack_cols && 2 * half <= 256) {
          t.z = 2 * half;
          t.w |= kUmmaStacked;
        }
        tnmax = std::max(tnmax, t.z);
      } else {
        c.um_thin_rmax = std::max(c.um_thin_rmax, std::min<int>(TM, (int)rows.size() - t.x));
      }
    c.n_tiles = (int)tl.size();
    c.um_tn = umma_tile_cols(std::max(tnmax, 32));
    const size_t need_b = (rows.size() + cols.size()) * sizeof(int2) + tl.size() * sizeof(int4) + clist.size() * sizeof(int) + 16;
    if (need_b > slot) return CK_ERR_OOM;
    c.d_rowdesc = base;
    c.d_coldesc = base + rows.size();
    c.d_um_tiles = reinterpret_cast<int4*>((reinterpret_cast<uintptr_t>(c.d_coldesc + cols.size()) + 15) & ~(uintptr_t)15);
    c.d_um_cols = reinterpret_cast<int*>(c.d_um_tiles + tl.size());
    cudaError_t e = cudaMemcpy(c.d_rowdesc, rows.data(), rows.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.d_coldesc, cols.data(), cols.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tl.empty()) e = cudaMemcpy(c.d_um_tiles, tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !clist.empty()) e = cudaMemcpy(c.d_um_cols, clist.data(), clist.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
    // the splits fill the SMs with tensor-core tiles (thin tiles take the same splits)
    c.um_cps = umma_cells_per_split(p.nc, std::max(c.um_ntc, 1), p.sm_count, p.tune.tc_ctas_per_sm);
    c.splits = (int)((p.nc + c.um_cps - 1) / c.um_cps);
    c.partial_doubles = (size_t)c.splits * std::max(c.n_tiles, 1) * TM * c.um_tn;
    if (c.partial_doubles > p.partials_cap) return CK_ERR_OOM;
    p.cplan_ready[mask] = true;
    return CK_OK;
  }
  // CUDA cores: the 64 x 64 output tiles holding a canonical (p, q)
  std::vector<int2> tiles;
  for (int m0 = 0; m0 < (int)rows.size(); m0 += BK_T)
    for (int n0 = 0; n0 < (int)cols.size(); n0 += BK_T) {
      bool any = false;
      for (int pp = m0; pp < std::min<int>(m0 + BK_T, (int)rows.size()) && !any; ++pp)
        for (int qq = n0; qq < std::min<int>(n0 + BK_T, (int)cols.size()) && !any; ++qq)
          any = canonical(rows[pp], cols[qq], mask, ms) != 0;
      if (any) tiles.push_back(make_int2(m0, n0));
    }
  c.n_tiles = (int)tiles.size();
  if ((rows.size() + cols.size() + tiles.size()) * sizeof(int2) > slot) return CK_ERR_OOM;
  c.d_rowdesc = base;
  c.d_coldesc = base + rows.size();
  c.d_tiles = base + rows.size() + cols.size();
  cudaError_t e = cudaMemcpy(c.d_rowdesc, rows.data(), rows.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c.d_coldesc, cols.data(), cols.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpy(c.d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  const int64_t per_split = (int64_t)std::max(c.n_tiles, 1) * BK_T * BK_T;
  int64_t splits = std::max<int64_t>(1, (int64_t)(4 * p.sm_count + c.n_tiles - 1) / std::max(c.n_tiles, 1));
  splits = std::min<int64_t>(splits, (int64_t)(p.partials_cap / per_split));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, p.nc / 128));
  if (splits < 1) return CK_ERR_OOM;
  c.splits = (int)splits;
  c.partial_doubles = (size_t)splits * per_split;
  p.cplan_ready[mask] = true;
  return CK_OK;
}

ck_status launch_contract(Plan& p, int mask, const float* w0, const float* bank, int64_t bstride,
                          double* sums, cudaStream_t st, const int* box) {
  const int64_t plane = (int64_t)p.grid.n[0] * p.grid.n[1];
  ck_status s = contract_prepare(p, mask);
  if (s != CK_OK) return s;
  const ContractPlan& c = p.cplan[mask];
  int* status = &p.dstate->status;
  if (c.use_reg) {
    cudaError_t e;
    {
    ProfScope ps(p, ST_CONTRACT, box ? 0.0 : 4.0 * (double)(p.ns + 1) * (double)p.nc, 0.0,
                 4.0 * (p.ns + 1) * (double)plane, box, st);
    e = launch_reg(p.ns, c.reg_maxn, w0, bank, bstride, p.nc, c.ctas, box, plane, p.partials, status, st);
    }
    if (e != cudaSuccess) return cuda_status(e);
    ProfScope ps2(p, ST_REDUCE, 8.0 * (double)c.partial_doubles, st);
    const int nkeep = (int)std::min<int64_t>(c.n_out_reg, p.n_multiset_total);
    reduce_reg_kernel<<<(nkeep + 127) / 128, 128, 0, st>>>(p.partials, c.ctas, c.n_out_reg, nkeep, sums);
    return cuda_status(cudaGetLastError());
  }
  if (c.n_tiles == 0) return CK_OK;
  if (c.use_tc) {
    cudaError_t e = cudaSuccess;
    const int nthin = c.n_tiles - c.um_ntc;
    // thin tiles beside the tensor-core kernel: on a second stream (forked
    // from and joined to st), with the tensor-core CTAs made large enough
    // that one per SM leaves room for a thin CTA
    const bool overlap = p.tune.tc_thin_overlap && nthin > 0 && c.um_ntc > 0;
    if (overlap) {
      if (!p.aux_stream) e = cudaStreamCreateWithFlags(&p.aux_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess && !p.aux_fork) e = cudaEventCreateWithFlags(&p.aux_fork, cudaEventDisableTiming);
      if (e == cudaSuccess && !p.aux_join) e = cudaEventCreateWithFlags(&p.aux_join, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_status(e);
    }
    {
      ProfScope ps(p, ST_CONTRACT, box ? 0.0 : 4.0 * (double)(p.ns + 1) * (double)p.nc * c.n_tiles, 0.0,
                   4.0 * (p.ns + 1) * (double)plane * c.n_tiles, box, st);
      cudaStream_t ts = st;
      size_t min_smem = 0;
      if (overlap) {
        e = cudaEventRecord(p.aux_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p.aux_stream, p.aux_fork, 0);
        ts = p.aux_stream;
        min_smem = (size_t)227 * 1024 - umma_thin_smem(p.ns, c.um_thin_rmax) - 2 * 1024;
      }
      if (e == cudaSuccess)
        e = launch_umma_thin(w0, bank, bstride, p.nc, p.ns, c.um_thin_rmax, c.d_rowdesc, c.rows, c.d_coldesc,
                             c.d_um_tiles, c.d_um_cols, c.um_ntc, nthin, c.n_tiles, c.um_tn, c.splits, box, plane,
                             p.partials, ts);
      if (e == cudaSuccess)
        e = launch_umma(c.um_tn, c.um_kind, w0, bank, bstride, p.nc, p.ns, c.d_rowdesc, c.rows, c.d_coldesc,
                        c.d_um_tiles, c.d_um_cols, c.um_ntc, c.n_tiles, c.splits, box, plane, p.absmax, p.partials,
                        status, st, min_smem);
      if (overlap) {
        const cudaError_t e2 = cudaEventRecord(p.aux_join, p.aux_stream);
        const cudaError_t e3 = e2 == cudaSuccess ? cudaStreamWaitEvent(st, p.aux_join, 0) : e2;
        if (e == cudaSuccess) e = e3;
      }
    }
    if (e != cudaSuccess) return cuda_status(e);
    ProfScope ps2(p, ST_REDUCE, 8.0 * (double)c.partial_doubles, st);
    return cuda_status(launch_umma_reduce(p.partials, c.splits, c.n_tiles, c.um_tn, c.d_um_tiles, c.d_um_cols,
                                          c.d_rowdesc, c.rows, c.d_coldesc, mask, p.ns, p.multiset_base, sums, st));
  }
  dim3 grid((unsigned)c.n_tiles, (unsigned)c.splits);
  {
  ProfScope ps(p, ST_CONTRACT, box ? 0.0 : 4.0 * (double)(p.ns + 1) * (double)p.nc, 0.0,
               4.0 * (p.ns + 1) * (double)plane, box, st);
  if (p.precision == CK_PREC_FP64_SUM)
    contract_blocked_kernel<double><<<grid, 256, 0, st>>>(w0, bank, bstride, p.nc, p.ns, c.d_rowdesc, c.rows,
                                                          c.d_coldesc, c.cols, c.d_tiles, c.n_tiles, box, plane,
                                                          p.partials);
  else
    contract_blocked_kernel<float><<<grid, 256, 0, st>>>(w0, bank, bstride, p.nc, p.ns, c.d_rowdesc, c.rows,
                                                         c.d_coldesc, c.cols, c.d_tiles, c.n_tiles, box, plane,
                                                         p.partials);
  }
  ProfScope ps2(p, ST_REDUCE, 8.0 * (double)c.partial_doubles, st);
  OrderBases B;
  for (int n = 0; n <= CK_MAX_ORDER; ++n) B.base[n] = p.multiset_base[n];
  const int64_t total = (int64_t)c.n_tiles * BK_T * BK_T;
  reduce_blocked_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      p.partials, c.splits, c.n_tiles, c.d_tiles, c.d_rowdesc, c.rows, c.d_coldesc, c.cols, mask, p.ns, B, sums);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// xi_n = num / (alpha^n den_raw) into dense symmetric tensors

// plain != 0: field sums with no denominator (Eq. 16): xi = num, den = 1.
__global__ void finalize_kernel(const double* __restrict__ sums, const double* __restrict__ den_raw,
                                const int* __restrict__ dmap, int64_t dense, int64_t mbase, int n, DevState* st,
                                double* __restrict__ xi, double* __restrict__ num, double* __restrict__ den,
                                int plain) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= dense) return;
  const int64_t r = mbase + dmap[d];
  if (plain) {
    num[d] = sums[r];
    xi[d] = sums[r];
    den[d] = 1.0;
    return;
  }
  const double alpha = st->alpha;
  double an = 1.0;
  for (int i = 0; i < n; ++i) an *= alpha;
  const double nu = sums[r];
  const double de = den_raw[r] * an;
  num[d] = nu;
  den[d] = de;
  if (de > 0.0) {
    xi[d] = nu / de;
  } else {
    xi[d] = __longlong_as_double(0x7ff8000000000000ll);
    set_status(&st->status, CK_ERR_ZERO_DENOM);
  }
}

void launch_finalize(const Plan& p, int mask, cudaStream_t st, bool plain) {
  ProfScope ps(p, ST_FINALIZE, 0.0, st);
  for (int n = 2; n <= p.max_order; ++n) {
    if (!((mask >> n) & 1)) continue;
    const int64_t dense = p.dense_elems[n];
    double* xi = p.dense + p.dense_base[n];
    double* num = p.dense + p.dense_total + p.dense_base[n];
    double* den = p.dense + 2 * p.dense_total + p.dense_base[n];
    finalize_kernel<<<(unsigned)((dense + 255) / 256), 256, 0, st>>>(
        p.sums, p.den_raw, p.dense_map + p.dense_base[n], dense, p.multiset_base[n], n, p.dstate, xi, num, den,
        plain ? 1 : 0);
  }
}

// host-side rank, used to build the dense -> multiset map
int64_t host_multiset_rank(const int* s, int k, int ns) { return multiset_rank(s, k, ns); }

}  // namespace ck

// ---------------------------------------------------------------------------
// ck_contract_static: the register contraction with its scratch (per-CTA
// partial sums and a status word) in a fixed file-scope device array instead
// of plan workspace, for callers that cannot allocate device memory.

namespace ck {
namespace {

constexpr int kStaticMaxCtas = 512;
constexpr int kStaticMaxOut = 152;  // register-kernel outputs: 16 shells, n <= 3
constexpr int kStaticMaxDevices = 64;
constexpr size_t kStaticDoubles = (size_t)kStaticMaxCtas * kStaticMaxOut + 32;

// Held by every GPU that loads this library, until the process exits.
static __device__ __align__(256) double g_contract_scratch[kStaticDoubles];

void* g_scratch_addr[kStaticMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Partials (CTA order, fixed) into each requested order's caller pointer;
// NaN everywhere if a device wait of the contraction gave up.
__global__ void static_reduce_kernel(const double* __restrict__ partials, int ctas, int nout, int ns, int maxn,
                                     const int* __restrict__ status, double* o2, double* o3, double* o4,
                                     double* o5) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double s = 0.0;
  for (int c = 0; c < ctas; ++c) s += partials[(int64_t)c * nout + o];
  if (*status != 0) s = __longlong_as_double(0x7ff8000000000000ll);
  const int n2 = ns, n3 = maxn >= 3 ? cmb(ns + 1, 2) : 0, n4 = maxn >= 4 ? cmb(ns + 2, 3) : 0;
  if (o < n2) { if (o2) o2[o] = s; return; }
  if (o < n2 + n3) { if (o3) o3[o - n2] = s; return; }
  if (o < n2 + n3 + n4) { if (o4) o4[o - n2 - n3] = s; return; }
  if (o5) o5[o - n2 - n3 - n4] = s;
}

}  // namespace
}  // namespace ck

using namespace ck;

extern "C" ck_status ck_contract_static(const float* w0, const float* bank, int64_t bank_stride, int64_t n_cells,
                                        int32_t n_shells, int32_t order_mask, double* const* sums, void* stream) {
  if (!w0 || !bank || !sums) return CK_ERR_BAD_POINTER;
  if (n_cells < 1 || n_shells < 1 || bank_stride < n_cells || (bank_stride % 4) != 0) return CK_ERR_ARG;
  if (order_mask == 0 || (order_mask & ~0x3c) != 0) return CK_ERR_ARG;
  const int maxn = max_order_in(order_mask);
  // the fixed scratch holds the register kernel's partial sums only
  if (!((n_shells <= 16 && maxn <= 3) || (n_shells <= 5 && maxn <= 5))) return CK_ERR_UNSUPPORTED;
  if (((uintptr_t)w0 & 15u) != 0 || ((uintptr_t)bank & 15u) != 0) return CK_ERR_BAD_POINTER;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return CK_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CK_ERR_CUDA;
  const int ctas = std::min(sms, kStaticMaxCtas);
  const int reg_maxn = maxn <= 3 ? 3 : 5;
  const int nout = reg_nout(n_shells, reg_maxn);
  if ((size_t)ctas * nout + 1 > kStaticDoubles - 31) return CK_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The array's device address, looked up with this device current.  Outside
  // stream capture it is looked up on every call, so that a context created
  // again (after cudaDeviceReset, say) never sees an address of the old one;
  // under capture the address of the last uncaptured call is used.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return CK_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_contract_scratch);
      if (e != cudaSuccess || !a) return CK_ERR_CUDA;
      g_scratch_addr[dev] = a;
    }
    base = g_scratch_addr[dev];
  }
  double* partials = static_cast<double*>(base);
  int* status = reinterpret_cast<int*>(partials + (size_t)ctas * nout);
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return CK_ERR_CUDA;
  cudaError_t e = launch_reg(n_shells, reg_maxn, w0, bank, bank_stride, n_cells, ctas, nullptr, 0, partials, status, st);
  if (e != cudaSuccess) return cuda_status(e);
  double* o[CK_MAX_ORDER + 1] = {nullptr};
  for (int n = 2; n <= CK_MAX_ORDER; ++n) o[n] = ((order_mask >> n) & 1) ? sums[n] : nullptr;
  static_reduce_kernel<<<(nout + 127) / 128, 128, 0, st>>>(partials, ctas, nout, n_shells, reg_maxn, status, o[2],
                                                           o[3], o[4], o[5]);
  return cuda_status(cudaGetLastError());
}

extern "C" ck_status ck_debug_force_timeout(int64_t ns) {
  const uint64_t v = ns > 0 ? (uint64_t)ns : 0;
  return cuda_status(cudaMemcpyToSymbol(g_force_timeout_ns, &v, sizeof(v)));
}
