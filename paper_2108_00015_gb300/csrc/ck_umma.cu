// ck_umma.cu -- the blocked product sums of Sec. 2.5 (Eqs. 11-13) on the
// fifth-generation tensor cores, for split-TF32 plans that keep the bank
// (orders >= 4 or more than 16 shells).
//
// The outputs are the entries T[p][q] = sum_r A_p(r) B_q(r) of the blocked
// product (A_p = W0 W_a W_b, B_q = W_c W_d, the same operand descriptors and
// canonical pairs as contract_blocked_kernel), in output tiles of 128 rows
// x TN columns held in tensor memory.  A CTA owns one tile and a range of
// cells (split-K):
//  * chunks of 32 cells are software-pipelined with one block barrier each:
//    after the barrier of chunk c, thread 0 issues the MMAs of chunk c - 1,
//    the CTA fetches the W values of chunk c + 1 with cp.async and builds
//    the operands of chunk c straight into the core-matrix layout of
//    ck_umma.cuh (double-buffered; a buffer is rebuilt once the commit of
//    the MMAs that read it has arrived on its mbarrier);
//  * every operand is split x = hi + lo, hi = x truncated to TF32 (exact),
//    lo = x - hi, and each 8-cell step issues hi*hi, hi*lo and lo*hi as
//    kind::tf32 MMAs (M = 128, N = TN, K = 8) accumulating in FP32 in
//    tensor memory; the dropped lo*lo term is below 2^-21 relative;
//  * every 8 chunks (256 cells) the accumulator is drained with tcgen05.ld
//    into FP32 registers of the CTA's 16 warps (warp w: lanes 32 (w % 4)..,
//    a quarter of the columns; the next chunk overwrites it), and each CTA
//    writes its FP32 register sums (at most 64 groups) as FP64 partials,
//    reduced over the splits in a fixed order.
// Waits are bounded: on a timeout the CTA sets CK_ERR_TIMEOUT, stops
// issuing, waits (bounded) for its own MMAs and frees its tensor memory.
#include <algorithm>
#include <vector>

#include "ck_device.cuh"
#include "ck_internal.h"
#include "ck_mma.cuh"
#include "ck_umma.cuh"

namespace ck {

namespace {

constexpr int UM_M = 128;
constexpr int UM_KC = 32;             // cells per chunk: 4 MMA k-steps of 8
constexpr int UM_GROUP = 8;           // chunks per tensor-memory accumulation (256 cells)
constexpr int UM_MAX_GROUPS = 64;     // groups per CTA (FP32 register sums)
constexpr int UM_WPITCH = UM_KC + 4;  // W staging row pitch (floats)
constexpr int UM_THREADS = 512;
constexpr int UM_WARPS = UM_THREADS / 32;

template <int TN>
struct UmmaShape {
  static_assert(TN % 32 == 0 && TN >= 32 && TN <= 256, "N of the MMA, four column quarters of 8s");
  static constexpr size_t a_bytes = (size_t)UM_M * UM_KC * sizeof(float);
  static constexpr size_t b_bytes = (size_t)TN * UM_KC * sizeof(float);
  static constexpr size_t stage_bytes = 2 * a_bytes + 2 * b_bytes;  // A hi, A lo, B hi, B lo
  static constexpr uint32_t ncols = TN <= 32 ? 32 : (TN <= 64 ? 64 : (TN <= 128 ? 128 : 256));
};

// W staging rows per buffer: W0, the ns shells, a row of ones and a row of zeros
__host__ __device__ constexpr int um_wrows(int ns) { return ns + 3; }

template <int TN>
size_t umma_smem(int ns) {
  using S = UmmaShape<TN>;
  return 2 * S::stage_bytes + (size_t)2 * um_wrows(ns) * UM_WPITCH * sizeof(float) +
         (size_t)(UM_M + TN) * sizeof(int4) + 64;
}

template <int TN>
__global__ void __launch_bounds__(UM_THREADS, 1)
    contract_umma_kernel(const float* __restrict__ w0, const float* __restrict__ bank, int64_t bstride, int64_t nc,
                         int ns, const int2* __restrict__ rowdesc, int rows, const int2* __restrict__ coldesc,
                         int cols, const int2* __restrict__ tiles, int ntiles, int64_t cells_per_split,
                         double* __restrict__ partials, int* status) {
  using S = UmmaShape<TN>;
  extern __shared__ __align__(1024) unsigned char um_smem[];
  unsigned char* stages = um_smem;  // [2][A hi | A lo | B hi | B lo]
  const int WR = um_wrows(ns);
  float* wsb = reinterpret_cast<float*>(um_smem + 2 * S::stage_bytes);  // [2][WR][WPITCH]
  int4* fa = reinterpret_cast<int4*>(wsb + 2 * WR * UM_WPITCH);         // [128] factor rows of A_p
  int4* fb = fa + UM_M;                                                  // [TN]  factor rows of B_q
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(fb + TN) + 15) & ~(uintptr_t)15);     // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  auto Ahi = [&](int b) { return reinterpret_cast<float*>(stages + b * S::stage_bytes); };
  auto Alo = [&](int b) { return reinterpret_cast<float*>(stages + b * S::stage_bytes + S::a_bytes); };
  auto Bhi = [&](int b) { return reinterpret_cast<float*>(stages + b * S::stage_bytes + 2 * S::a_bytes); };
  auto Blo = [&](int b) {
    return reinterpret_cast<float*>(stages + b * S::stage_bytes + 2 * S::a_bytes + S::b_bytes);
  };
  auto Ws = [&](int b) { return wsb + b * WR * UM_WPITCH; };
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int2 tile = tiles[blockIdx.x];
  // each operand row is the product of three staged rows: A_p = W0 W_a W_b, B_q = 1 W_c W_d,
  // with the ones row for an absent factor and the zeros row for a padding row
  const int ONE = ns + 1, ZERO = ns + 2;
  for (int i = tid; i < UM_M; i += UM_THREADS) {
    const int p = tile.x + i;
    const int2 d = p < rows ? rowdesc[p] : make_int2(-2, -2);
    fa[i] = d.x == -2 ? make_int4(ZERO, ONE, ONE, 0)
                      : make_int4(0, d.x >= 0 ? 1 + d.x : ONE, d.y >= 0 ? 1 + d.y : ONE, 0);
  }
  for (int i = tid; i < TN; i += UM_THREADS) {
    const int q = tile.y + i;
    const int2 d = q < cols ? coldesc[q] : make_int2(-2, -2);
    fb[i] = d.x == -2 ? make_int4(ZERO, ONE, ONE, 0)
                      : make_int4(ONE, d.x >= 0 ? 1 + d.x : ONE, d.y >= 0 ? 1 + d.y : ONE, 0);
  }
  for (int i = tid; i < 2 * UM_KC; i += UM_THREADS) {  // constant rows of both staging buffers
    float* w = wsb + (i / UM_KC) * WR * UM_WPITCH;
    w[ONE * UM_WPITCH + i % UM_KC] = 1.0f;
    w[ZERO * UM_WPITCH + i % UM_KC] = 0.0f;
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, S::ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  const int64_t beg = (int64_t)blockIdx.y * cells_per_split;
  const int64_t end = std::min<int64_t>(nc, beg + cells_per_split);
  const int nch = end > beg ? (int)((end - beg + UM_KC - 1) / UM_KC) : 0;
  // W values of chunk c into staging buffer b: 16-byte copies of 4 cells,
  // zero past `end` (w0, the bank rows, bstride and beg are multiples of 4 floats)
  auto stage = [&](int c, int b) {
    const int64_t c0 = beg + (int64_t)c * UM_KC;
    float* dst = Ws(b);
    for (int idx = tid; idx < (ns + 1) * (UM_KC / 4); idx += UM_THREADS) {  // rows 0..ns only
      const int a = idx / (UM_KC / 4), j = idx - a * (UM_KC / 4);
      const int64_t cell = c0 + 4 * j;
      const int64_t left = end - cell;
      const int n = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
      const float* src = a == 0 ? w0 : bank + (int64_t)(a - 1) * bstride;
      cp_async16n(dst + a * UM_WPITCH + 4 * j, n > 0 ? (const void*)(src + cell) : (const void*)w0, n);
    }
  };
  // operands of one chunk: warp w builds row-cores w, w + 16, .. of A and B,
  // all 8 cell-cores of each (8 rows x 4 cells, 128 contiguous bytes per core)
  const int rr = lane >> 2, kk = lane & 3;
  auto build_rows = [&](const float* w, const int4 f, float* hi, float* lo, int R, int r8) {
    const float* x0 = w + f.x * UM_WPITCH + kk;
    const float* x1 = w + f.y * UM_WPITCH + kk;
    const float* x2 = w + f.z * UM_WPITCH + kk;
    float* h = hi + r8 * 32 + lane;
    float* l = lo + r8 * 32 + lane;
#pragma unroll
    for (int k4 = 0; k4 < UM_KC / 4; ++k4) {
      const float v = x0[4 * k4] * x1[4 * k4] * x2[4 * k4];
      const float vh = __uint_as_float(tf32_trunc(v));
      h[k4 * (R / 8) * 32] = vh;  // core (r8, k4) of an R-row block
      l[k4 * (R / 8) * 32] = v - vh;
    }
  };
  auto build = [&](int b) {
    const float* w = Ws(b);
    for (int r8 = warp; r8 < UM_M / 8; r8 += UM_WARPS) build_rows(w, fa[8 * r8 + rr], Ahi(b), Alo(b), UM_M, r8);
    for (int r8 = warp; r8 < TN / 8; r8 += UM_WARPS) build_rows(w, fb[8 * r8 + rr], Bhi(b), Blo(b), TN, r8);
  };
  // thread 0: the 12 MMAs of chunk c (operand buffer c & 1), then one commit
  auto issue = [&](int c) {
    const int b = c & 1;
    constexpr uint32_t idesc = umma_idesc_tf32(UM_M, TN);
    constexpr uint32_t a_lbo = UM_M / 8 * 128, b_lbo = TN / 8 * 128;
    const uint32_t ahs = smem_u32(Ahi(b)), als = smem_u32(Alo(b));
    const uint32_t bhs = smem_u32(Bhi(b)), bls = smem_u32(Blo(b));
    const bool first = c % UM_GROUP == 0;
#pragma unroll
    for (int s = 0; s < UM_KC / 8; ++s) {
      const uint32_t ao = 2 * s * a_lbo, bo = 2 * s * b_lbo;  // two core columns (8 cells) per step
      const uint64_t dah = umma_desc(ahs + ao, a_lbo, 128), dal = umma_desc(als + ao, a_lbo, 128);
      const uint64_t dbh = umma_desc(bhs + bo, b_lbo, 128), dbl = umma_desc(bls + bo, b_lbo, 128);
      umma_tf32(tbase, dah, dbh, idesc, !(first && s == 0));
      umma_tf32(tbase, dah, dbl, idesc, true);
      umma_tf32(tbase, dal, dbh, idesc, true);
    }
    umma_commit(&bar[b]);
  };

  // register sums: warp w drains lanes 32 (w % 4).. of columns (w / 4) TN / 4 ..
  constexpr int QTR = TN / 4;
  float mid[QTR];
#pragma unroll
  for (int j = 0; j < QTR; ++j) mid[j] = 0.0f;
  const uint32_t lane_base = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * QTR);

  bool ok = true;
  int issued = 0;  // chunks whose MMAs have been committed
  if (nch > 0) stage(0, 0);
  cp_async_commit();
  for (int c = 0; c <= nch; ++c) {
    cp_async_wait<0>();
    if (__syncthreads_or(!ok)) break;  // W of chunk c landed, operands of chunk c - 1 built
    if (c >= 1) {
      if (tid == 0) {
        tc_fence_after();
        issue(c - 1);
      }
      issued = c;
    }
    if (c + 1 < nch) stage(c + 1, (c + 1) & 1);
    cp_async_commit();
    if (c < nch) {
      // buffer c & 1 was read by the MMAs of chunk c - 2
      if (c >= 2) ok = mbar_wait(&bar[c & 1], (uint32_t)((c - 2) >> 1) & 1u, status);
      if (ok) build(c & 1);
      fence_async_shared();  // the operands, written by this thread, for the tensor cores
    }
    // chunk c - 1 closes a group: drain the accumulator once its MMAs are done
    // (tcgen05.ld is warp-collective: the warp decides together)
    if (c >= 1 && ((c - 1) % UM_GROUP == UM_GROUP - 1 || c - 1 == nch - 1)) {
      if (ok) ok = mbar_wait(&bar[(c - 1) & 1], (uint32_t)((c - 1) >> 1) & 1u, status);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (ok) {
        tc_fence_after();
#pragma unroll
        for (int j0 = 0; j0 < QTR; j0 += 8) {
          float v[8];
          tmem_ld8(lane_base + j0, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) mid[j0 + j] += v[j];
        }
        tc_fence_before();
      }
    }
  }
  // after a timeout: the MMAs already committed must finish before tensor memory is freed
  if (!ok && tid == 0 && issued > 0)
    mbar_wait(&bar[(issued - 1) & 1], (uint32_t)((issued - 1) >> 1) & 1u, status);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tbase, S::ncols);
  double* out = partials + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (int64_t)(UM_M * TN);
  const int row = 32 * (warp & 3) + lane;
  const int col0 = (warp >> 2) * QTR;
#pragma unroll
  for (int j = 0; j < QTR; ++j) out[row * TN + col0 + j] = (double)mid[j];
}

// Which order (and multiset) a (row, column) pair computes: the same rule as
// the blocked kernel's reduction (canonical pairs of the requested orders).
__device__ inline int umma_canonical(int2 rd, int2 cd, int mask, int* ms) {
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

__device__ inline int64_t umma_rank(const int* s, int k, int ns) {
  int64_t r = 0;
  int prev = 0;
  for (int t = 0; t < k; ++t) {
    for (int v = prev; v < s[t]; ++v) {
      const int n = ns - v + (k - t - 1) - 1, kk = k - t - 1;
      int64_t c = 1;
      for (int i = 1; i <= kk; ++i) c = c * (n - kk + i) / i;
      r += c;
    }
    prev = s[t];
  }
  return r;
}

struct UmmaBases {
  int64_t base[CK_MAX_ORDER + 1];
};

__global__ void reduce_umma_kernel(const double* __restrict__ partials, int splits, int ntiles, int tn,
                                   const int2* __restrict__ tiles, const int2* __restrict__ rowdesc, int rows,
                                   const int2* __restrict__ coldesc, int cols, int mask, int ns, UmmaBases B,
                                   double* __restrict__ out) {
  const int64_t per = (int64_t)UM_M * tn;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ntiles * per) return;
  const int tile = (int)(t / per);
  const int pq = (int)(t - (int64_t)tile * per);
  const int p = tiles[tile].x + pq / tn, q = tiles[tile].y + pq % tn;
  if (p >= rows || q >= cols) return;
  int ms[4];
  const int n = umma_canonical(rowdesc[p], coldesc[q], mask, ms);
  if (!n) return;
  double s = 0.0;
  for (int sp = 0; sp < splits; ++sp) s += partials[((int64_t)sp * ntiles + tile) * per + pq];
  out[B.base[n] + umma_rank(ms, n - 1, ns)] = s;
}

template <int TN>
cudaError_t launch_umma_t(const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns, const int2* rowdesc,
                          int rows, const int2* coldesc, int cols, const int2* tiles, int ntiles, int splits,
                          int64_t cps, double* partials, int* status, cudaStream_t st) {
  const size_t sm = umma_smem<TN>(ns);
  cudaError_t e = cudaFuncSetAttribute(contract_umma_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ntiles, (unsigned)splits);
  contract_umma_kernel<TN><<<grid, UM_THREADS, sm, st>>>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, cols,
                                                         tiles, ntiles, cps, partials, status);
  return cudaGetLastError();
}

}  // namespace

int umma_tile_cols(int cols) {
  if (cols <= 32) return 32;
  if (cols <= 64) return 64;
  if (cols <= 128) return 128;
  if (cols <= 160) return 160;
  return 256;
}

int umma_tile_rows() { return UM_M; }

// Cells per split: whole chunks, at most UM_MAX_GROUPS accumulation groups.
int64_t umma_cells_per_split(int64_t nc, int ntiles, int sm_count) {
  const int64_t cap = (int64_t)UM_MAX_GROUPS * UM_GROUP * UM_KC;
  int64_t splits = std::max<int64_t>(1, (2 * (int64_t)sm_count + ntiles - 1) / std::max(ntiles, 1));
  int64_t cps = (nc + splits - 1) / splits;
  cps = std::min(cps, cap);
  cps = (cps + UM_KC - 1) / UM_KC * UM_KC;
  return std::max<int64_t>(cps, UM_KC);
}

cudaError_t launch_umma(int tn, const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns,
                        const int2* rowdesc, int rows, const int2* coldesc, int cols, const int2* tiles, int ntiles,
                        int splits, int64_t cps, double* partials, int* status, cudaStream_t st) {
  switch (tn) {
    case 32: return launch_umma_t<32>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, cols, tiles, ntiles, splits, cps, partials, status, st);
    case 64: return launch_umma_t<64>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, cols, tiles, ntiles, splits, cps, partials, status, st);
    case 128: return launch_umma_t<128>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, cols, tiles, ntiles, splits, cps, partials, status, st);
    case 160: return launch_umma_t<160>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, cols, tiles, ntiles, splits, cps, partials, status, st);
    case 256: return launch_umma_t<256>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, cols, tiles, ntiles, splits, cps, partials, status, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_umma_reduce(const double* partials, int splits, int ntiles, int tn, const int2* tiles,
                               const int2* rowdesc, int rows, const int2* coldesc, int cols, int mask, int ns,
                               const int64_t* bases, double* out, cudaStream_t st) {
  UmmaBases B;
  for (int n = 0; n <= CK_MAX_ORDER; ++n) B.base[n] = bases[n];
  const int64_t total = (int64_t)ntiles * UM_M * tn;
  reduce_umma_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(partials, splits, ntiles, tn, tiles, rowdesc,
                                                                      rows, coldesc, cols, mask, ns, B, out);
  return cudaGetLastError();
}

}  // namespace ck
