// ck_umma.cu -- the blocked product sums of Sec. 2.5 (Eqs. 11-13) on the
// fifth-generation tensor cores, for split-TF32 plans that keep the bank
// (orders >= 4 or more than 16 shells).
//
// The outputs are the entries T[p][q] = sum_r A_p(r) B_q(r) of the blocked
// product (A_p = W0 W_a W_b, B_q = W_c W_d, the same operand descriptors and
// canonical pairs as contract_blocked_kernel).  A tile is 128 consecutive
// rows and a list of the columns that hold a canonical pair with one of
// them (rows sorted by their last factor, so the late row tiles of order 5
// need few columns), MMA N = the list length rounded up to 32; it is
// accumulated in tensor memory.  A CTA owns one tile and a
// range of cells (split-K), walked in chunks of 32 cells by three kinds of
// warps that meet only on mbarriers (no block barrier per chunk):
//  * warp 0 stages the W values of up to 8 chunks at once (W0 and the bank
//    rows, 1 KB each) with cp.async.bulk copies into two staging buffers
//    (a copy of 128 bytes per row and chunk kept the copy engine busy
//    longer than the tensor cores);
//  * warps 2..17 build the split operands of a chunk: warp w owns A rows
//    32 (w % 4) .. + 31 (its tensor-memory lane quarter) for a quarter of
//    the chunk's cells and writes them with tcgen05.st into one of three A
//    stages in tensor memory; together the sixteen warps write B into the
//    matching shared-memory stage, in the no-swizzle K-major core layout of
//    ck_umma.cuh (each warp's B addresses are fixed for the CTA and kept in
//    registers; operands of padding rows and columns are zeroed once);
//  * one thread of warp 1 issues, per chunk, 12 kind::tf32 MMAs (M = 128,
//    N = TN, K = 8; A from tensor memory, B from shared memory) and commits
//    them to the stage's mbarrier, which frees the stage for the builders.
// Every operand is split x = hi + lo, hi = x truncated to TF32 (exact),
// lo = x - hi, and each 8-cell step issues hi*hi, hi*lo and lo*hi,
// accumulating in FP32 in tensor memory; the dropped lo*lo term is below
// 2^-21 relative.  Every 8 chunks (256 cells) close an accumulation group:
// the builder warps drain its accumulator with tcgen05.ld into FP32
// registers while the MMAs of the next group run into the second
// accumulator (two accumulators where tensor memory holds them, else one,
// drained before the next group starts).  Each CTA writes its FP32
// register sums (at most 64 groups) as FP64 partials, reduced over the
// splits in a fixed order.
// Waits are bounded: on a timeout a warp sets CK_ERR_TIMEOUT and stops;
// before tensor memory is freed the MMA thread waits (bounded) for its last
// commit and the staging warp for its copies in flight.
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
constexpr int UM_NA = 3;              // operand stages
constexpr int UM_MAX_NW = 3;          // W staging buffers (at most)
constexpr int UM_BWARPS = 16;         // builder warps: four per tensor-memory lane quarter
constexpr int UM_THREADS = 32 * (2 + UM_BWARPS);
constexpr int UM_ACOLS = 2 * UM_KC;   // tensor-memory columns of one A stage: hi | lo

template <int TN>
struct UmmaShape {
  static_assert(TN % 32 == 0 && TN >= 32 && TN <= 256, "N of the MMA, four column quarters of 8s");
  static constexpr size_t b_bytes = (size_t)TN * UM_KC * sizeof(float);
  static constexpr size_t stage_bytes = 2 * b_bytes;  // B hi | B lo
  // two accumulators when they fit next to the A stages in 512 columns
  static constexpr int nacc = 2 * TN + UM_NA * UM_ACOLS <= 512 ? 2 : 1;
  static constexpr int a_col0 = nacc * TN;
  static constexpr int used = a_col0 + UM_NA * UM_ACOLS;
  static_assert(used <= 512, "tensor memory");
  static constexpr uint32_t ncols = used <= 32 ? 32 : (used <= 64 ? 64 : (used <= 128 ? 128 : (used <= 256 ? 256 : 512)));
  static constexpr int quarter = TN / 4;  // accumulator columns drained by one warp (at most)
};

// W staging rows per buffer: W0, the ns shells, a row of ones and a row of zeros
__host__ __device__ constexpr int um_wrows(int ns) { return ns + 3; }

// W staging row pitch (floats) for wch chunks per buffer: 16-byte rows
// whose 16-byte index is 1 mod 8, so eight lanes reading eight different
// rows at the same cell hit eight different bank groups
__host__ __device__ constexpr int um_wpitch(int wch) { return wch * UM_KC + 4; }

template <int TN>
size_t umma_smem(int ns, int nw, int wch) {
  using S = UmmaShape<TN>;
  return UM_NA * S::stage_bytes + (size_t)nw * um_wrows(ns) * um_wpitch(wch) * sizeof(float) +
         (size_t)TN * sizeof(int4) + (2 * UM_MAX_NW + 2 * UM_NA + 4) * sizeof(uint64_t) + 16;
}

// Staging buffers and chunks per buffer: the longest bulk copies that fit
// (8 chunks = 1 KB per row), double-buffered.
template <int TN>
bool umma_staging(int ns, size_t limit, int* nw, int* wch) {
  for (int c = 8; c >= 1; c /= 2)
    if (umma_smem<TN>(ns, 2, c) <= limit) {
      *nw = 2;
      *wch = c;
      return true;
    }
  return false;
}

template <int TN>
__global__ void __launch_bounds__(UM_THREADS, 1)
    contract_umma_kernel(const float* __restrict__ w0, const float* __restrict__ bank, int64_t bstride, int64_t nc,
                         int ns, int nw, int wch, const int2* __restrict__ rowdesc, int rows, const int2* __restrict__ coldesc,
                         const int4* __restrict__ tiles, const int* __restrict__ collist, int ntiles,
                         int64_t cells_per_split, double* __restrict__ partials, int* status) {
  using S = UmmaShape<TN>;
  // every shared-memory pointer derives from the array by pointer arithmetic
  // (no integer round trip), so the compiler emits shared-space accesses
  extern __shared__ __align__(1024) unsigned char um_smem[];
  unsigned char* smem = um_smem;
  unsigned char* stages = smem;  // [UM_NA][B hi | B lo]
  const int WR = um_wrows(ns);
  const int wp = um_wpitch(wch);
  float* wsb = reinterpret_cast<float*>(smem + UM_NA * S::stage_bytes);  // [nw][WR][wp]
  int4* fb = reinterpret_cast<int4*>(wsb + nw * WR * wp);                 // [TN] factor rows of B_q
  uint64_t* bar = reinterpret_cast<uint64_t*>(fb + TN);
  uint64_t* wfull = bar;                     // [UM_MAX_NW] W staged (bulk-copy bytes)
  uint64_t* wempty = wfull + UM_MAX_NW;      // [UM_MAX_NW] W read by the builder warps
  uint64_t* sfull = wempty + UM_MAX_NW;      // [UM_NA] operands of a stage written
  uint64_t* sempty = sfull + UM_NA;          // [UM_NA] MMAs of a stage complete (commit)
  uint64_t* afull = sempty + UM_NA;          // [2] MMAs of a group complete (commit)
  uint64_t* aempty = afull + 2;              // [2] accumulator drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(aempty + 2);
  auto Bhi = [&](int s) { return reinterpret_cast<float*>(stages + s * S::stage_bytes); };
  auto Blo = [&](int s) { return reinterpret_cast<float*>(stages + s * S::stage_bytes + S::b_bytes); };
  auto Ws = [&](int b) { return wsb + b * WR * wp; };
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // tile: rows tile.x .. + 127, columns collist[tile.y + i] for i < tile.w,
  // MMA N = tn = tile.z (a multiple of 32, at most TN)
  const int4 tile = tiles[blockIdx.x];
  const int tn = tile.z;
  // each operand row is the product of staged rows: A_p = W0 W_a W_b, B_q = W_c W_d,
  // with the ones row for an absent factor and the zeros row for a padding row
  const int ONE = ns + 1, ZERO = ns + 2;
  for (int i = tid; i < TN; i += UM_THREADS) {
    const int2 d = i < tile.w ? coldesc[collist[tile.y + i]] : make_int2(-2, -2);
    fb[i] = d.x == -2 ? make_int4(ZERO, ONE, 0, 0) : make_int4(d.x >= 0 ? 1 + d.x : ONE, d.y >= 0 ? 1 + d.y : ONE, 0, 0);
  }
  const int wcells = wch * UM_KC;  // cells per staging buffer
  for (int i = tid; i < nw * wcells; i += UM_THREADS) {  // constant rows of every staging buffer
    float* w = Ws(i / wcells);
    w[ONE * wp + i % wcells] = 1.0f;
    w[ZERO * wp + i % wcells] = 0.0f;
  }
  if (tid == 0) {
    for (int i = 0; i < UM_MAX_NW; ++i) {
      mbar_init(&wfull[i], 1);
      mbar_init(&wempty[i], UM_BWARPS);
    }
    for (int i = 0; i < UM_NA; ++i) {
      mbar_init(&sfull[i], UM_BWARPS);
      mbar_init(&sempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], UM_BWARPS);
    }
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
  const int ngroups = (nch + UM_GROUP - 1) / UM_GROUP;
  constexpr int NACC = S::nacc;
  constexpr uint32_t FULL = 0xFFFFFFFFu;

  if (warp == 0) {
    // ---- staging: W0 and the bank rows of chunks f wch .. f wch + wch - 1
    // (fill f) into buffer f % nw
    bool ok = true;
    int staged = 0;
    const int nfill = (nch + wch - 1) / wch;
    for (int f = 0; f < nfill; ++f) {
      const int b = f % nw;
      if (f >= nw) ok = mbar_wait(&wempty[b], (uint32_t)(f / nw - 1) & 1u, status);
      if (!__all_sync(FULL, ok)) break;
      const int64_t c0 = beg + (int64_t)f * wcells;
      const int valid = (int)std::min<int64_t>(wcells, end - c0);
      float* dst = Ws(b);
      if (valid == wcells) {  // 16-byte aligned rows (c0 is a multiple of 32 cells)
        if (lane == 0) mbar_arrive_expect_tx(&wfull[b], (uint32_t)((ns + 1) * wcells * sizeof(float)));
        __syncwarp();
        for (int a = lane; a <= ns; a += 32)
          bulk_g2s(dst + a * wp, (a == 0 ? w0 : bank + (int64_t)(a - 1) * bstride) + c0,
                   (uint32_t)(wcells * sizeof(float)), &wfull[b]);
      } else {  // the last, partial fill: plain copies, zeros past the end
        for (int i = lane; i < (ns + 1) * wcells; i += 32) {
          const int a = i / wcells, k = i - a * wcells;
          const float* src = a == 0 ? w0 : bank + (int64_t)(a - 1) * bstride;
          dst[a * wp + k] = k < valid ? src[c0 + k] : 0.0f;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&wfull[b]);
      }
      staged = f + 1;
    }
    // no copy may still be landing in shared memory when the CTA ends
    for (int f = std::max(0, staged - nw); f < staged; ++f) mbar_wait(&wfull[f % nw], (uint32_t)(f / nw) & 1u, status);
  } else if (warp == 1) {
    // ---- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_tf32(UM_M, tn);
      const uint32_t b_lbo = (uint32_t)(tn / 8 * 128);
      bool ok = true;
      int last = -1;
      for (int c = 0; c < nch; ++c) {
        const int g = c / UM_GROUP, a = g % NACC, s = c % UM_NA;
        const bool first = c % UM_GROUP == 0;
        if (first && g >= NACC) ok = mbar_wait(&aempty[a], (uint32_t)(g / NACC - 1) & 1u, status);
        if (ok) ok = mbar_wait(&sfull[s], (uint32_t)(c / UM_NA) & 1u, status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dt = tbase + (uint32_t)(a * TN);
        const uint32_t ah = tbase + (uint32_t)(S::a_col0 + s * UM_ACOLS), al = ah + UM_KC;
        const uint32_t bhs = smem_u32(Bhi(s)), bls = smem_u32(Blo(s));
#pragma unroll
        for (int k = 0; k < UM_KC / 8; ++k) {
          const uint32_t bo = 2 * k * b_lbo;  // two core columns (8 cells) per step
          const uint64_t dbh = umma_desc(bhs + bo, b_lbo, 128), dbl = umma_desc(bls + bo, b_lbo, 128);
          umma_tf32_ts(dt, ah + 8 * k, dbh, idesc, !(first && k == 0));
          umma_tf32_ts(dt, ah + 8 * k, dbl, idesc, true);
          umma_tf32_ts(dt, al + 8 * k, dbh, idesc, true);
        }
        umma_commit(&sempty[s]);
        if (c % UM_GROUP == UM_GROUP - 1 || c == nch - 1) umma_commit(&afull[a]);
        last = c;
      }
      // every MMA issued must be complete before tensor memory is freed
      if (last >= 0) mbar_wait(&sempty[last % UM_NA], (uint32_t)(last / UM_NA) & 1u, status);
    }
  } else {
    // ---- operand build and accumulator drains
    const int bw = warp - 2;          // 0..15
    const int qd = warp & 3;          // tensor-memory lane quarter
    const int pt = bw >> 2;           // A: cells 8 pt .. 8 pt + 7; drains: column quarter pt
    const int m = 32 * qd + lane;     // A row of this thread
    int fx, fy, fz;
    {
      const int p = tile.x + m;
      const int2 d = p < rows ? rowdesc[p] : make_int2(-2, -2);
      fx = d.x == -2 ? ZERO : 0;
      fy = d.x >= 0 ? 1 + d.x : ONE;
      fz = d.y >= 0 ? 1 + d.y : ONE;
    }
    const bool a_live = __any_sync(FULL, tile.x + m < rows);  // a lane quarter of padding rows stays zero
    const uint32_t tq = tbase + ((uint32_t)(32 * qd) << 16);
    const int qc = tn / 4;  // accumulator columns this warp drains (a multiple of 8)
    // B items of this warp, it = bw + 16 j: 8 columns (row core r8 = it / 2) x
    // 4 cell cores (4 (it % 2) .. + 3); lane: column 8 r8 + rr, cell core kc
    constexpr int IT = (TN / 4 + UM_BWARPS - 1) / UM_BWARPS;
    const int rr = lane & 7, kq = lane >> 3;
    int bu[IT], bv[IT];
    bool bl_live[IT], b_any[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
      const int it = bw + UM_BWARPS * j;
      const int r8 = it >> 1, kc = 4 * (it & 1) + kq;
      b_any[j] = it < tn / 4;
      bl_live[j] = b_any[j] && 8 * r8 < tile.w;  // uniform over the warp
      const int4 f = b_any[j] ? fb[8 * r8 + rr] : make_int4(ZERO, ONE, 0, 0);
      bu[j] = f.x * wp + 4 * kc;
      bv[j] = f.y * wp + 4 * kc;
    }
    auto b_off = [&](int j) {
      const int it = bw + UM_BWARPS * j;
      return ((4 * (it & 1) + kq) * (tn / 8) + (it >> 1)) * 32 + rr * 4;  // core (r8, kc), row rr
    };
    // zero, once, the operands that no chunk writes
    if (!a_live) {
      const uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int s = 0; s < UM_NA; ++s) {
        const uint32_t ta = tq + (uint32_t)(S::a_col0 + s * UM_ACOLS + 8 * pt);
        tmem_st8(ta, z);
        tmem_st8(ta + UM_KC, z);
      }
      tmem_wait_st();
    }
#pragma unroll
    for (int j = 0; j < IT; ++j)
      if (b_any[j] && !bl_live[j])
        for (int s = 0; s < UM_NA; ++s) {
          *reinterpret_cast<float4*>(Bhi(s) + b_off(j)) = make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(Blo(s) + b_off(j)) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    float mid[S::quarter];
#pragma unroll
    for (int j = 0; j < S::quarter; ++j) mid[j] = 0.0f;
    auto drain = [&](int g) -> bool {
      const int a = g % NACC;
      bool ok = mbar_wait(&afull[a], (uint32_t)(g / NACC) & 1u, status);
      if (!__all_sync(FULL, ok)) return false;
      tc_fence_after();
#pragma unroll
      for (int j0 = 0; j0 < S::quarter; j0 += 8) {
        if (j0 < qc) {  // uniform over the warp
          float v[8];
          tmem_ld8(tq + (uint32_t)(a * TN + pt * qc + j0), v);
#pragma unroll
          for (int j = 0; j < 8; ++j) mid[j0 + j] += v[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[a]);
      return true;
    };
    // group g is drained after building chunk drain_at(g): half a group
    // later with two accumulators, else before the next group needs it
    auto drain_at = [&](int g) {
      return NACC == 2 ? (g + 1) * UM_GROUP + UM_GROUP / 2 - 1 : (g + 1) * UM_GROUP + UM_NA - 1;
    };
    bool ok = true;
    int next = 0;  // next group to drain
    for (int c = 0; c < nch && ok; ++c) {
      const int fl = c / wch, b = fl % nw, s = c % UM_NA;
      if (c % wch == 0) ok = mbar_wait(&wfull[b], (uint32_t)(fl / nw) & 1u, status);
      if (ok && c >= UM_NA) ok = mbar_wait(&sempty[s], (uint32_t)(c / UM_NA - 1) & 1u, status);
      if (!__all_sync(FULL, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const float* w = Ws(b) + (c % wch) * UM_KC;
      if (a_live) {  // A row m, cells 8 pt .. 8 pt + 7: hi and lo into the stage's tensor-memory columns
        const float4* x0 = reinterpret_cast<const float4*>(w + fx * wp + 8 * pt);
        const float4* x1 = reinterpret_cast<const float4*>(w + fy * wp + 8 * pt);
        const float4* x2 = reinterpret_cast<const float4*>(w + fz * wp + 8 * pt);
        const float4 a0 = x0[0], a1 = x1[0], a2 = x2[0], c0 = x0[1], c1 = x1[1], c2 = x2[1];
        const float v[8] = {a0.x * a1.x * a2.x, a0.y * a1.y * a2.y, a0.z * a1.z * a2.z, a0.w * a1.w * a2.w,
                            c0.x * c1.x * c2.x, c0.y * c1.y * c2.y, c0.z * c1.z * c2.z, c0.w * c1.w * c2.w};
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          hi[e] = tf32_trunc(v[e]);
          lo[e] = __float_as_uint(v[e] - __uint_as_float(hi[e]));
        }
        const uint32_t ta = tq + (uint32_t)(S::a_col0 + s * UM_ACOLS + 8 * pt);
        tmem_st8(ta, hi);
        tmem_st8(ta + UM_KC, lo);
      }
      // B: all loads of this warp's items first, then products, splits and stores
      float4 u[IT], v[IT];
#pragma unroll
      for (int j = 0; j < IT; ++j)
        if (bl_live[j]) {
          u[j] = *reinterpret_cast<const float4*>(w + bu[j]);
          v[j] = *reinterpret_cast<const float4*>(w + bv[j]);
        }
      float* bh = Bhi(s);
      float* bl = Blo(s);
#pragma unroll
      for (int j = 0; j < IT; ++j)
        if (bl_live[j]) {
          const float p0 = u[j].x * v[j].x, p1 = u[j].y * v[j].y, p2 = u[j].z * v[j].z, p3 = u[j].w * v[j].w;
          const float4 h = make_float4(__uint_as_float(tf32_trunc(p0)), __uint_as_float(tf32_trunc(p1)),
                                       __uint_as_float(tf32_trunc(p2)), __uint_as_float(tf32_trunc(p3)));
          const int off = b_off(j);
          *reinterpret_cast<float4*>(bh + off) = h;
          *reinterpret_cast<float4*>(bl + off) = make_float4(p0 - h.x, p1 - h.y, p2 - h.z, p3 - h.w);
        }
      if (a_live) tmem_wait_st();
      fence_async_shared();  // the B operands, for the tensor cores
      tc_fence_before();     // the A operands (tcgen05.st), for the MMA thread
      __syncwarp();
      if (lane == 0) {
        if (c % wch == wch - 1 || c == nch - 1) mbar_arrive(&wempty[b]);  // the fill is read
        mbar_arrive(&sfull[s]);
      }
      while (ok && next < ngroups && c >= drain_at(next)) ok = drain(next++);
    }
    while (ok && next < ngroups) ok = drain(next++);
    // per-CTA partials: row m, this warp's quarter of the columns
    double* out = partials + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (int64_t)(UM_M * TN);
#pragma unroll
    for (int j = 0; j < S::quarter; ++j)
      if (j < qc) out[m * TN + pt * qc + j] = (double)mid[j];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tbase, S::ncols);
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
                                   const int4* __restrict__ tiles, const int* __restrict__ collist,
                                   const int2* __restrict__ rowdesc, int rows, const int2* __restrict__ coldesc,
                                   int mask, int ns, UmmaBases B, double* __restrict__ out) {
  const int64_t per = (int64_t)UM_M * tn;  // partials per tile: 128 rows of pitch tn
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ntiles * per) return;
  const int tile = (int)(t / per);
  const int pq = (int)(t - (int64_t)tile * per);
  const int4 tl = tiles[tile];
  const int p = tl.x + pq / tn, ci = pq % tn;
  if (p >= rows || ci >= tl.w) return;
  const int q = collist[tl.y + ci];
  int ms[4];
  const int n = umma_canonical(rowdesc[p], coldesc[q], mask, ms);
  if (!n) return;
  double s = 0.0;
  for (int sp = 0; sp < splits; ++sp) s += partials[((int64_t)sp * ntiles + tile) * per + pq];
  out[B.base[n] + umma_rank(ms, n - 1, ns)] = s;
}

template <int TN>
cudaError_t launch_umma_t(const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns, const int2* rowdesc,
                          int rows, const int2* coldesc, const int4* tiles, const int* collist, int ntiles,
                          int splits, int64_t cps, double* partials, int* status, cudaStream_t st) {
  int nw = 0, wch = 0;
  if (!umma_staging<TN>(ns, (size_t)227 * 1024, &nw, &wch)) return cudaErrorInvalidValue;
  const size_t sm = umma_smem<TN>(ns, nw, wch);
  cudaError_t e = cudaFuncSetAttribute(contract_umma_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ntiles, (unsigned)splits);
  contract_umma_kernel<TN><<<grid, UM_THREADS, sm, st>>>(w0, bank, bstride, nc, ns, nw, wch, rowdesc, rows, coldesc,
                                                         tiles, collist, ntiles, cps, partials, status);
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

// Cells per split: whole accumulation groups (256 cells), at most UM_MAX_GROUPS.
int64_t umma_cells_per_split(int64_t nc, int ntiles, int sm_count) {
  const int64_t cap = (int64_t)UM_MAX_GROUPS * UM_GROUP * UM_KC;
  int64_t splits = std::max<int64_t>(1, (2 * (int64_t)sm_count + ntiles - 1) / std::max(ntiles, 1));
  int64_t cps = (nc + splits - 1) / splits;
  cps = std::min(cps, cap);
  cps = (cps + UM_GROUP * UM_KC - 1) / (UM_GROUP * UM_KC) * (UM_GROUP * UM_KC);  // whole staging fills
  return std::max<int64_t>(cps, UM_GROUP * UM_KC);
}

cudaError_t launch_umma(int tn, const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns,
                        const int2* rowdesc, int rows, const int2* coldesc, const int4* tiles, const int* collist,
                        int ntiles, int splits, int64_t cps, double* partials, int* status, cudaStream_t st) {
  switch (tn) {
    case 32: return launch_umma_t<32>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, tiles, collist, ntiles, splits, cps, partials, status, st);
    case 64: return launch_umma_t<64>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, tiles, collist, ntiles, splits, cps, partials, status, st);
    case 128: return launch_umma_t<128>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, tiles, collist, ntiles, splits, cps, partials, status, st);
    case 160: return launch_umma_t<160>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, tiles, collist, ntiles, splits, cps, partials, status, st);
    case 256: return launch_umma_t<256>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, tiles, collist, ntiles, splits, cps, partials, status, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_umma_reduce(const double* partials, int splits, int ntiles, int tn, const int4* tiles,
                               const int* collist, const int2* rowdesc, int rows, const int2* coldesc, int mask,
                               int ns, const int64_t* bases, double* out, cudaStream_t st) {
  UmmaBases B;
  for (int n = 0; n <= CK_MAX_ORDER; ++n) B.base[n] = bases[n];
  const int64_t total = (int64_t)ntiles * UM_M * tn;
  reduce_umma_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(partials, splits, ntiles, tn, tiles, collist,
                                                                      rowdesc, rows, coldesc, mask, ns, B, out);
  return cudaGetLastError();
}

}  // namespace ck
