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
// accumulated in tensor memory.  A CTA owns one tile and a range of cells
// (split-K), walked in chunks of KC cells (KC = 64 for TN <= 160, else 32)
// by three kinds of warps that meet only on mbarriers (no block barrier per
// chunk), 320 threads:
//  * warp 0 stages the W values of 256 cells at a time (W0 and the bank
//    rows, 1 KB each) with cp.async.bulk copies into two staging buffers
//    (a copy of 128 bytes per row and chunk kept the copy engine busy
//    longer than the tensor cores);
//  * warps 2..9 (eight builders, two per tensor-memory lane quarter) build
//    the split operands of a chunk: warp w owns A rows 32 (w % 4) .. + 31
//    (its lane quarter) for half of the chunk's cells and writes them with
//    tcgen05.st into one of NA A stages in tensor memory (NA = 2 for TN =
//    128 and 160, else 3); together the eight warps write B into the
//    matching shared-memory stage, in the no-swizzle K-major core layout of
//    ck_umma.cuh (each warp's B addresses are fixed for the CTA and kept in
//    registers; operands of padding rows and columns are zeroed once);
//  * one thread of warp 1 issues, per chunk, 3 KC / 8 kind::tf32 MMAs (24
//    for KC = 64; M = 128, N = TN, K = 8; A from tensor memory, B from
//    shared memory) and commits them to the stage's mbarrier, which frees
//    the stage for the builders.
// Every operand is split x = hi + lo, hi = x truncated to TF32 (exact),
// lo = x - hi, and each 8-cell step issues hi*hi, hi*lo and lo*hi,
// accumulating in FP32 in tensor memory; the dropped lo*lo term is below
// 2^-21 relative.  Every 256 cells (256 / KC chunks) close an accumulation
// group: the builder warps drain its accumulator with tcgen05.ld into FP32
// registers while the MMAs of the next group run into the second
// accumulator (two accumulators where tensor memory holds them next to the
// A stages, else one, drained before the next group starts).  Each CTA
// writes its FP32 register sums (at most 64 groups) as FP64 partials,
// reduced over the splits in a fixed order.
// Waits are bounded: on a timeout a warp sets CK_ERR_TIMEOUT and stops;
// before tensor memory is freed the MMA thread waits (bounded) for its last
// commit and the staging warp for its copies in flight.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ck_device.cuh"
#include "ck_internal.h"
#include "ck_mma.cuh"
#include "ck_umma.cuh"

namespace ck {

namespace {

constexpr int UM_M = 128;
constexpr int UM_GCELLS = 256;        // cells per tensor-memory accumulation group
constexpr int UM_MAX_GROUPS = 64;     // groups per CTA (FP32 register sums)
constexpr int UM_MAX_NA = 3;          // operand stages (at most)
constexpr int UM_MAX_NW = 2;          // W staging buffers
constexpr int UM_BWARPS = 8;          // builder warps: two per tensor-memory lane quarter
constexpr int UM_THREADS = 32 * (2 + UM_BWARPS);

// Operand kinds of the split product: TF32 (kind::tf32, K = 8 per MMA),
// BF16 and FP16 (kind::f16, K = 16 per MMA, two values per 32-bit
// tensor-memory column and per 4 bytes of a shared-memory core row).
constexpr int UM_TF32 = 0, UM_BF16 = 1, UM_FP16 = 2;

// FP16 operands are scaled by powers of two: each factor W by 2^-e with
// max |W| <= 2^e, and every product by 2^14, so |A_p|, |B_q| <= 2^14 stay
// inside the FP16 range; the partials are divided by the same exact scales.
constexpr float UM_FP16_HEAD = 16384.0f;

// Per tile width TN and kind: cells per chunk KC (64, or 32 where the TF32
// operand stages would not fit), operand stages NA, accumulators in tensor
// memory (two where they fit next to the A stages in 512 columns, else one).
template <int TN, int KIND = UM_TF32>
struct UmmaShape {
  static_assert(TN % 32 == 0 && TN >= 32 && TN <= 256, "N of the MMA, two column halves of 16s");
  static constexpr bool F16 = KIND != UM_TF32;
  static constexpr int EB = F16 ? 2 : 4;                       // operand element bytes
  static constexpr int KC = F16 ? 64 : (TN <= 160 ? 64 : 32);
  static constexpr int KS = F16 ? 16 : 8;                      // cells per MMA k-step
  static constexpr int NK = KC / KS;                           // MMA k-steps per chunk
  static constexpr int ACOLS = F16 ? KC : 2 * KC;              // A stage columns: hi | lo
  static constexpr int NA = F16 ? (TN == 256 ? 2 : 3) : ((TN == 128 || TN == 160) ? 2 : 3);
  static constexpr int G = UM_GCELLS / KC;                     // chunks per group
  static constexpr size_t b_bytes = (size_t)TN * KC * EB;
  static constexpr size_t stage_bytes = 2 * b_bytes;           // B hi | B lo
  static constexpr int nacc = 2 * TN + NA * ACOLS <= 512 ? 2 : 1;
  static constexpr int a_col0 = nacc * TN;
  static constexpr int used = a_col0 + NA * ACOLS;
  static_assert(NA <= UM_MAX_NA && used <= 512, "tensor memory");
  static constexpr uint32_t ncols = used <= 32 ? 32 : (used <= 64 ? 64 : (used <= 128 ? 128 : (used <= 256 ? 256 : 512)));
  static constexpr int half = TN / 2;     // accumulator columns drained by one warp (at most)
  static constexpr int UN = TN / 32;      // B units per warp (at most): 2 TN / 8 units over 8 warps
};

// W staging rows per buffer: W0, the ns shells, a row of ones and a row of zeros
__host__ __device__ constexpr int um_wrows(int ns) { return ns + 3; }

// W staging row pitch (floats) for `cells` cells per buffer: 16-byte rows
// whose 16-byte index is 1 mod 8, so eight lanes reading eight different
// rows at the same cell hit eight different bank groups
__host__ __device__ constexpr int um_wpitch(int cells) { return cells + 4; }

template <int TN, int KIND>
size_t umma_smem(int ns, int wcells) {
  using S = UmmaShape<TN, KIND>;
  return S::NA * S::stage_bytes + (size_t)UM_MAX_NW * um_wrows(ns) * um_wpitch(wcells) * sizeof(float) +
         (size_t)TN * sizeof(int4) + (size_t)TN * sizeof(float) +
         (2 * UM_MAX_NW + 2 * UM_MAX_NA + 4) * sizeof(uint64_t) + 16;
}

// Cells per staging buffer: the longest bulk copies that fit (256 cells =
// 1 KB per row), a whole number of chunks, double-buffered.
template <int TN, int KIND>
int umma_wcells(int ns, size_t limit) {
  using S = UmmaShape<TN, KIND>;
  for (int c = 256; c >= S::KC; c /= 2)
    if (umma_smem<TN, KIND>(ns, c) <= limit) return c;
  return 0;
}

// Power-of-two scale of one staged factor row for FP16 operands: 2^-e with
// max |row| <= 2^e (maxima as float bits in absmax; row 0 = W0, 1 + s =
// shell s); 1 for the ones row, for an all-zero row and for other kinds.
template <int KIND>
__device__ __forceinline__ float um_factor_scale(const unsigned* absmax, int row, int ones_row) {
  if (KIND != UM_FP16 || row >= ones_row) return 1.0f;
  const float mx = __uint_as_float(absmax[row]);
  if (!(mx > 0.0f) || !(mx < 3.0e38f)) return 1.0f;
  int e;
  frexpf(mx, &e);
  return ldexpf(1.0f, -e);
}

// Two 16-bit values (a in the low half) of the operand kind, from FP32.
template <int KIND>
__device__ __forceinline__ uint32_t um_pack2(float a, float b) {
  if constexpr (KIND == UM_BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// x = hi + lo + r with hi, lo of the operand kind (round to nearest): the
// packed pairs of hi and lo for (a, b).
template <int KIND>
__device__ __forceinline__ void um_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = um_pack2<KIND>(a, b);
  float ha, hb;
  if constexpr (KIND == UM_BF16) {
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&hi);
    ha = __low2float(h);
    hb = __high2float(h);
  } else {
    const __half2 h = *reinterpret_cast<const __half2*>(&hi);
    ha = __low2float(h);
    hb = __high2float(h);
  }
  lo = um_pack2<KIND>(a - ha, b - hb);
}

// Tiles of at most 64 columns fit two CTAs per SM (96 registers, under
// 100 KB of shared memory each).
template <int TN, int KIND>
__global__ void __launch_bounds__(UM_THREADS, TN <= 64 ? 2 : 1)
    contract_umma_kernel(const float* __restrict__ w0, const float* __restrict__ bank, int64_t bstride, int64_t nc,
                         int ns, int wcells, const int2* __restrict__ rowdesc, int rows,
                         const int2* __restrict__ coldesc, const int4* __restrict__ tiles,
                         const int* __restrict__ collist, int ntiles, const int* __restrict__ box, int64_t plane,
                         const unsigned* __restrict__ absmax, double* __restrict__ partials, int* status) {
  using S = UmmaShape<TN, KIND>;
  constexpr int KC = S::KC, NA = S::NA, G = S::G, NACC = S::nacc;
  constexpr int nw = UM_MAX_NW;
  // every shared-memory pointer derives from the array by pointer arithmetic
  // (no integer round trip), so the compiler emits shared-space accesses
  extern __shared__ __align__(1024) unsigned char um_smem[];
  unsigned char* stages = um_smem;  // [NA][B hi | B lo]
  const int WR = um_wrows(ns);
  const int wp = um_wpitch(wcells);
  const int wch = wcells / KC;  // chunks per staging buffer
  float* wsb = reinterpret_cast<float*>(um_smem + NA * S::stage_bytes);  // [nw][WR][wp]
  int4* fb = reinterpret_cast<int4*>(wsb + nw * WR * wp);                 // [TN] factor rows of B_q
  float* fsc = reinterpret_cast<float*>(fb + TN);                         // [TN] scale of B_q (FP16)
  uint64_t* bar = reinterpret_cast<uint64_t*>(fsc + TN);
  uint64_t* wfull = bar;                     // [nw] W staged (bulk-copy bytes)
  uint64_t* wempty = wfull + UM_MAX_NW;      // [nw] W read by the builder warps
  uint64_t* sfull = wempty + UM_MAX_NW;      // [NA] operands of a stage written
  uint64_t* sempty = sfull + UM_MAX_NA;      // [NA] MMAs of a stage complete (commit)
  uint64_t* afull = sempty + UM_MAX_NA;      // [2] MMAs of a group complete (commit)
  uint64_t* aempty = afull + 2;              // [2] accumulator drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(aempty + 2);
  auto Bhi = [&](int s) { return reinterpret_cast<float*>(stages + s * S::stage_bytes); };
  auto Blo = [&](int s) { return reinterpret_cast<float*>(stages + s * S::stage_bytes + S::b_bytes); };
  auto BhiB = [&](int s) { return stages + s * S::stage_bytes; };
  auto BloB = [&](int s) { return stages + s * S::stage_bytes + S::b_bytes; };
  auto Ws = [&](int b) { return wsb + b * WR * wp; };
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // tile: rows tile.x .. + 127, columns collist[tile.y + i] for i < cnt,
  // MMA N = tn = tile.z (a multiple of 32, at most TN); a stacked tile holds
  // B's hi part in MMA columns 0 .. tnb - 1 and its lo part in tnb ..
  const int4 tile = tiles[blockIdx.x];
  const int tn = tile.z;
  const bool stk = (tile.w & kUmmaStacked) != 0;
  const int cnt = tile.w & (kUmmaStacked - 1);
  const int tnb = stk ? tn / 2 : tn;  // columns whose products the builders form
  // each operand row is the product of staged rows: A_p = W0 W_a W_b, B_q = W_c W_d,
  // with the ones row for an absent factor and the zeros row for a padding row
  const int ONE = ns + 1, ZERO = ns + 2;
  for (int i = tid; i < TN; i += UM_THREADS) {
    const int2 d = i < cnt ? coldesc[collist[tile.y + i]] : make_int2(-2, -2);
    fb[i] = d.x == -2 ? make_int4(ZERO, ONE, 0, 0) : make_int4(d.x >= 0 ? 1 + d.x : ONE, d.y >= 0 ? 1 + d.y : ONE, 0, 0);
    fsc[i] = d.x == -2 ? 1.0f
                       : um_factor_scale<KIND>(absmax, d.x >= 0 ? 1 + d.x : ONE, ONE) *
                             um_factor_scale<KIND>(absmax, d.y >= 0 ? 1 + d.y : ONE, ONE) *
                             (KIND == UM_FP16 ? UM_FP16_HEAD : 1.0f);
  }
  for (int i = tid; i < nw * wcells; i += UM_THREADS) {  // constant rows of every staging buffer
    float* w = Ws(i / wcells);
    w[ONE * wp + i % wcells] = 1.0f;
    w[ZERO * wp + i % wcells] = 0.0f;
  }
  if (tid == 0) {
    for (int i = 0; i < nw; ++i) {
      mbar_init(&wfull[i], 1);
      mbar_init(&wempty[i], UM_BWARPS);
    }
    for (int i = 0; i < NA; ++i) {
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

  // this split's part of the visited cells: whole accumulation groups
  int64_t beg, end;
  split_cells(box_cells(box, plane, nc), gridDim.y, UM_GCELLS, blockIdx.y, &beg, &end);
  const int nch = end > beg ? (int)((end - beg + KC - 1) / KC) : 0;
  const int ngroups = (nch + G - 1) / G;
  constexpr uint32_t FULL = 0xFFFFFFFFu;

  if (warp == 0) {
    // ---- staging: W0 and the bank rows of fill f (chunks f wch ..) into buffer f % nw
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
      const uint32_t idesc = KIND == UM_TF32 ? umma_idesc_tf32(UM_M, tn) : umma_idesc_f16(UM_M, tn, KIND == UM_BF16);
      const uint32_t b_lbo = (uint32_t)(tn / 8 * 128);
      bool ok = true;
      int last = -1;
      for (int c = 0; c < nch; ++c) {
        const int g = c / G, a = g % NACC, s = c % NA;
        const bool first = c % G == 0;
        if (first && g >= NACC) ok = mbar_wait(&aempty[a], (uint32_t)(g / NACC - 1) & 1u, status);
        if (ok) ok = mbar_wait(&sfull[s], (uint32_t)(c / NA) & 1u, status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dt = tbase + (uint32_t)(a * TN);
        const uint32_t ah = tbase + (uint32_t)(S::a_col0 + s * S::ACOLS), al = ah + S::ACOLS / 2;
        const uint32_t bhs = smem_u32(Bhi(s)), bls = smem_u32(Blo(s));
#pragma unroll
        for (int k = 0; k < S::NK; ++k) {
          // two core columns per step (8 cells of TF32, 16 of BF16 / FP16);
          // A advances by 8 tensor-memory columns either way
          const uint32_t bo = 2 * k * b_lbo;
          const uint64_t dbh = umma_desc(bhs + bo, b_lbo, 128), dbl = umma_desc(bls + bo, b_lbo, 128);
          if (stk) {  // B = [hi | lo]: hi*hi, hi*lo, lo*hi and lo*lo in two MMAs
            if constexpr (KIND == UM_TF32) {
              umma_tf32_ts(dt, ah + 8 * k, dbh, idesc, !(first && k == 0));
              umma_tf32_ts(dt, al + 8 * k, dbh, idesc, true);
            } else {
              umma_f16_ts(dt, ah + 8 * k, dbh, idesc, !(first && k == 0));
              umma_f16_ts(dt, al + 8 * k, dbh, idesc, true);
            }
          } else if constexpr (KIND == UM_TF32) {
            umma_tf32_ts(dt, ah + 8 * k, dbh, idesc, !(first && k == 0));
            umma_tf32_ts(dt, ah + 8 * k, dbl, idesc, true);
            umma_tf32_ts(dt, al + 8 * k, dbh, idesc, true);
          } else {
            umma_f16_ts(dt, ah + 8 * k, dbh, idesc, !(first && k == 0));
            umma_f16_ts(dt, ah + 8 * k, dbl, idesc, true);
            umma_f16_ts(dt, al + 8 * k, dbh, idesc, true);
          }
        }
        umma_commit(&sempty[s]);
        if (c % G == G - 1 || c == nch - 1) umma_commit(&afull[a]);
        last = c;
      }
      // every MMA issued must be complete before tensor memory is freed
      if (last >= 0) mbar_wait(&sempty[last % NA], (uint32_t)(last / NA) & 1u, status);
    }
  } else {
    // ---- operand build and accumulator drains
    const int bw = warp - 2;          // 0..7
    const int qd = warp & 3;          // tensor-memory lane quarter
    const int hf = bw >> 2;           // A: cells hf KC/2 .. + KC/2 - 1; drains: column half hf
    const int m = 32 * qd + lane;     // A row of this thread
    int ax, ay, az;                   // staged-row offsets of the three factors of A row m
    float asc = 1.0f;                 // FP16: scale of A row m
    {
      const int p = tile.x + m;
      const int2 d = p < rows ? rowdesc[p] : make_int2(-2, -2);
      ax = (d.x == -2 ? ZERO : 0) * wp + hf * (KC / 2);
      ay = (d.x >= 0 ? 1 + d.x : ONE) * wp + hf * (KC / 2);
      az = (d.y >= 0 ? 1 + d.y : ONE) * wp + hf * (KC / 2);
      if (KIND == UM_FP16 && d.x != -2)
        asc = um_factor_scale<KIND>(absmax, 0, ONE) * um_factor_scale<KIND>(absmax, d.x >= 0 ? 1 + d.x : ONE, ONE) *
              um_factor_scale<KIND>(absmax, d.y >= 0 ? 1 + d.y : ONE, ONE) * UM_FP16_HEAD;
    }
    const bool a_live = __any_sync(FULL, tile.x + m < rows);  // a lane quarter of padding rows stays zero
    const uint32_t tq = tbase + ((uint32_t)(32 * qd) << 16);
    const int hc = tn / 2;  // accumulator columns this warp drains (a multiple of 16)
    // B units of this warp, u = bw + 8 j: row core r8 = u / 2, cells
    // (u % 2) KC/2 .. + KC/2 - 1, in items of 16 cells; lane: column
    // 8 r8 + rr, cell core 4 item + kq of the unit
    const int rr = lane & 7, kq = lane >> 3;
    int bu[S::UN], bv[S::UN];
    float bsc[S::UN];  // FP16: scale of this lane's column of each unit
    bool b_live[S::UN], b_any[S::UN];
#pragma unroll
    for (int j = 0; j < S::UN; ++j) {
      const int u = bw + UM_BWARPS * j;
      const int r8 = u >> 1;
      b_any[j] = u < tnb / 4;
      b_live[j] = b_any[j] && 8 * r8 < cnt;  // uniform over the warp
      const int4 f = b_any[j] ? fb[8 * r8 + rr] : make_int4(ZERO, ONE, 0, 0);
      bu[j] = f.x * wp + (u & 1) * (KC / 2) + 4 * kq;
      bv[j] = f.y * wp + (u & 1) * (KC / 2) + 4 * kq;
      bsc[j] = b_any[j] ? fsc[8 * r8 + rr] : 1.0f;
    }
    // where the lo part of a B item goes: the lo buffer, or (stacked tile)
    // tnb columns = tnb / 8 cores further in the hi buffer
    auto BloF = [&](int s) { return stk ? Bhi(s) + (tnb / 8) * 32 : Blo(s); };
    auto BloB2 = [&](int s) { return stk ? BhiB(s) + (tnb / 8) * 128 : BloB(s); };
    // floats: core (r8, kc), row rr of a B stage (kc = 4 item + kq)
    auto b_off = [&](int j, int item) {
      const int u = bw + UM_BWARPS * j;
      const int kc = (u & 1) * (KC / 8) + 4 * item + kq;
      return (kc * (tn / 8) + (u >> 1)) * 32 + rr * 4;
    };
    // bytes, 16-bit kinds: 8 cells per core row, this lane's 4 cells in half of it
    auto b_off16 = [&](int j, int item) {
      const int u = bw + UM_BWARPS * j;
      const int kc = (u & 1) * (KC / 16) + 2 * item + (kq >> 1);
      return (kc * (tn / 8) + (u >> 1)) * 128 + rr * 16 + (kq & 1) * 8;
    };
    // zero, once, the operands that no chunk writes
    if (!a_live) {
      const uint32_t z[8] = {};
      constexpr int hcols = S::ACOLS / 4;  // hi columns of this warp's half of the cells
      for (int s = 0; s < NA; ++s)
        for (int i = 0; i < hcols / 8; ++i) {
          const uint32_t ta = tq + (uint32_t)(S::a_col0 + s * S::ACOLS + hf * hcols + 8 * i);
          tmem_st8(ta, z);
          tmem_st8(ta + S::ACOLS / 2, z);
        }
      tmem_wait_st();
    }
#pragma unroll
    for (int j = 0; j < S::UN; ++j)
      if (b_any[j] && !b_live[j])
        for (int s = 0; s < NA; ++s)
          for (int i = 0; i < KC / 32; ++i) {
            if constexpr (KIND == UM_TF32) {
              *reinterpret_cast<float4*>(Bhi(s) + b_off(j, i)) = make_float4(0.f, 0.f, 0.f, 0.f);
              *reinterpret_cast<float4*>(BloF(s) + b_off(j, i)) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
              *reinterpret_cast<uint2*>(BhiB(s) + b_off16(j, i)) = make_uint2(0u, 0u);
              *reinterpret_cast<uint2*>(BloB2(s) + b_off16(j, i)) = make_uint2(0u, 0u);
            }
          }
    float mid[S::half];
#pragma unroll
    for (int j = 0; j < S::half; ++j) mid[j] = 0.0f;
    auto drain = [&](int g) -> bool {
      const int a = g % NACC;
      bool ok = mbar_wait(&afull[a], (uint32_t)(g / NACC) & 1u, status);
      if (!__all_sync(FULL, ok)) return false;
      tc_fence_after();
#pragma unroll
      for (int j0 = 0; j0 < S::half; j0 += 16) {
        if (j0 < hc) {  // uniform over the warp
          float v[16];
          tmem_ld16(tq + (uint32_t)(a * TN + hf * hc + j0), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) mid[j0 + j] += v[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[a]);
      return true;
    };
    // group g is drained after building chunk drain_at(g): half a group
    // later with two accumulators, else before the next group needs it
    auto drain_at = [&](int g) { return NACC == 2 ? (g + 1) * G + G / 2 - 1 : (g + 1) * G + NA - 1; };
    bool ok = true;
    int next = 0;  // next group to drain
    for (int c = 0; c < nch && ok; ++c) {
      const int fl = c / wch, b = fl % nw, s = c % NA;
      if (c % wch == 0) ok = mbar_wait(&wfull[b], (uint32_t)(fl / nw) & 1u, status);
      if (ok && c >= NA) ok = mbar_wait(&sempty[s], (uint32_t)(c / NA - 1) & 1u, status);
      if (!__all_sync(FULL, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const float* w = Ws(b) + (c % wch) * KC;
      float* bh = Bhi(s);
      float* bl = BloF(s);
#pragma unroll
      for (int i = 0; i < KC / 32; ++i) {  // 16 cells per item
        if (a_live && KIND != UM_TF32) {  // A row m, 16 cells: packed hi and lo pairs
          float v[16];
#pragma unroll
          for (int h8 = 0; h8 < 2; ++h8) {
            const int o = 16 * i + 8 * h8;
            const float4 x0 = *reinterpret_cast<const float4*>(w + ax + o);
            const float4 x1 = *reinterpret_cast<const float4*>(w + ay + o);
            const float4 x2 = *reinterpret_cast<const float4*>(w + az + o);
            const float4 y0 = *reinterpret_cast<const float4*>(w + ax + o + 4);
            const float4 y1 = *reinterpret_cast<const float4*>(w + ay + o + 4);
            const float4 y2 = *reinterpret_cast<const float4*>(w + az + o + 4);
            v[8 * h8 + 0] = x0.x * x1.x * x2.x;
            v[8 * h8 + 1] = x0.y * x1.y * x2.y;
            v[8 * h8 + 2] = x0.z * x1.z * x2.z;
            v[8 * h8 + 3] = x0.w * x1.w * x2.w;
            v[8 * h8 + 4] = y0.x * y1.x * y2.x;
            v[8 * h8 + 5] = y0.y * y1.y * y2.y;
            v[8 * h8 + 6] = y0.z * y1.z * y2.z;
            v[8 * h8 + 7] = y0.w * y1.w * y2.w;
          }
          if constexpr (KIND == UM_FP16) {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] *= asc;
          }
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) um_split2<KIND>(v[2 * e], v[2 * e + 1], hi[e], lo[e]);
          const uint32_t ta = tq + (uint32_t)(S::a_col0 + s * S::ACOLS + (hf * (KC / 2) + 16 * i) / 2);
          tmem_st8(ta, hi);
          tmem_st8(ta + S::ACOLS / 2, lo);
        }
        if (a_live && KIND == UM_TF32) {  // A row m, 8 cells at a time: hi and lo into the stage's tensor-memory columns
#pragma unroll
          for (int h8 = 0; h8 < 2; ++h8) {
            const int o = 16 * i + 8 * h8;
            const float4 x0 = *reinterpret_cast<const float4*>(w + ax + o);
            const float4 x1 = *reinterpret_cast<const float4*>(w + ay + o);
            const float4 x2 = *reinterpret_cast<const float4*>(w + az + o);
            const float4 y0 = *reinterpret_cast<const float4*>(w + ax + o + 4);
            const float4 y1 = *reinterpret_cast<const float4*>(w + ay + o + 4);
            const float4 y2 = *reinterpret_cast<const float4*>(w + az + o + 4);
            const float v[8] = {x0.x * x1.x * x2.x, x0.y * x1.y * x2.y, x0.z * x1.z * x2.z, x0.w * x1.w * x2.w,
                                y0.x * y1.x * y2.x, y0.y * y1.y * y2.y, y0.z * y1.z * y2.z, y0.w * y1.w * y2.w};
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              hi[e] = tf32_trunc(v[e]);
              lo[e] = __float_as_uint(v[e] - __uint_as_float(hi[e]));
            }
            const uint32_t ta = tq + (uint32_t)(S::a_col0 + s * S::ACOLS + hf * (KC / 2) + o);
            tmem_st8(ta, hi);
            tmem_st8(ta + KC, lo);
          }
        }
        // this warp's B items of the same 16 cells: all loads, then products, splits and stores
        float4 u4[S::UN], v4[S::UN];
#pragma unroll
        for (int j = 0; j < S::UN; ++j)
          if (b_live[j]) {
            u4[j] = *reinterpret_cast<const float4*>(w + bu[j] + 16 * i);
            v4[j] = *reinterpret_cast<const float4*>(w + bv[j] + 16 * i);
          }
#pragma unroll
        for (int j = 0; j < S::UN; ++j)
          if (b_live[j]) {
            float p0 = u4[j].x * v4[j].x, p1 = u4[j].y * v4[j].y, p2 = u4[j].z * v4[j].z, p3 = u4[j].w * v4[j].w;
            if constexpr (KIND == UM_TF32) {
              const float4 h = make_float4(__uint_as_float(tf32_trunc(p0)), __uint_as_float(tf32_trunc(p1)),
                                           __uint_as_float(tf32_trunc(p2)), __uint_as_float(tf32_trunc(p3)));
              const int off = b_off(j, i);
              *reinterpret_cast<float4*>(bh + off) = h;
              *reinterpret_cast<float4*>(bl + off) = make_float4(p0 - h.x, p1 - h.y, p2 - h.z, p3 - h.w);
            } else {
              if constexpr (KIND == UM_FP16) {
                p0 *= bsc[j];
                p1 *= bsc[j];
                p2 *= bsc[j];
                p3 *= bsc[j];
              }
              uint2 h, l;
              um_split2<KIND>(p0, p1, h.x, l.x);
              um_split2<KIND>(p2, p3, h.y, l.y);
              const int off = b_off16(j, i);
              *reinterpret_cast<uint2*>(BhiB(s) + off) = h;
              *reinterpret_cast<uint2*>(BloB2(s) + off) = l;
            }
          }
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
    // per-CTA partials: row m, this warp's half of the columns
    double* out = partials + ((int64_t)blockIdx.y * ntiles + blockIdx.x) * (int64_t)(UM_M * TN);
#pragma unroll
    for (int j = 0; j < S::half; ++j)
      if (j < hc) {
        double v = (double)mid[j];
        if constexpr (KIND == UM_FP16) v /= (double)asc * (double)fsc[stk ? j : hf * hc + j];  // exact powers of two
        out[m * TN + hf * hc + j] = v;
      }
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

// One warp per partial element (tile, row, column): lane l sums the splits
// l, l + 32, .. in order, then a fixed shuffle tree adds the lanes, so the
// result is the same from run to run.
__global__ void reduce_umma_kernel(const double* __restrict__ partials, int splits, int ntiles, int tn,
                                   const int4* __restrict__ tiles, const int* __restrict__ collist,
                                   const int2* __restrict__ rowdesc, int rows, const int2* __restrict__ coldesc,
                                   int mask, int ns, UmmaBases B, double* __restrict__ out) {
  const int64_t per = (int64_t)UM_M * tn;  // partials per tile: 128 rows of pitch tn
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)ntiles * per) return;
  const int tile = (int)(t / per);
  const int pq = (int)(t - (int64_t)tile * per);
  const int4 tl = tiles[tile];
  const int p = tl.x + pq / tn, ci = pq % tn;  // row and column of the partial
  const int cnt = tl.w & (kUmmaStacked - 1);
  if (p >= rows || ci >= cnt) return;
  const int q = collist[tl.y + ci];
  int ms[4];
  const int n = umma_canonical(rowdesc[p], coldesc[q], mask, ms);
  if (!n) return;
  // a stacked tile's lo half sits tl.z / 2 columns to the right
  const int lo = (tl.w & kUmmaStacked) ? tl.z / 2 : 0;
  double s = 0.0;
  for (int sp = lane; sp < splits; sp += 32) {
    const double* pt = partials + ((int64_t)sp * ntiles + tile) * per + pq;
    s += lo ? pt[0] + pt[lo] : pt[0];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) out[B.base[n] + umma_rank(ms, n - 1, ns)] = s;
}

template <int TN, int KIND>
cudaError_t launch_umma_t(const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns, const int2* rowdesc,
                          int rows, const int2* coldesc, const int4* tiles, const int* collist, int ntc, int ntiles,
                          int splits, const int* box, int64_t plane, const unsigned* absmax, double* partials,
                          int* status, cudaStream_t st, size_t min_smem) {
  if (ntc == 0) return cudaSuccess;
  const int wcells = umma_wcells<TN, KIND>(ns, (size_t)227 * 1024);
  if (wcells == 0) return cudaErrorInvalidValue;
  // the kernel uses umma_smem bytes; a larger request only limits residency
  const size_t sm = std::min<size_t>(std::max(umma_smem<TN, KIND>(ns, wcells), min_smem), (size_t)227 * 1024);
  cudaError_t e =
      cudaFuncSetAttribute(contract_umma_kernel<TN, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ntc, (unsigned)splits);  // tiles 0 .. ntc - 1; partials pitched by all ntiles
  contract_umma_kernel<TN, KIND><<<grid, UM_THREADS, sm, st>>>(w0, bank, bstride, nc, ns, wcells, rowdesc, rows,
                                                               coldesc, tiles, collist, ntiles, box, plane, absmax,
                                                               partials, status);
  return cudaGetLastError();
}

// Largest |value| of W0 (row 0) and of each bank row (1 + s), as float bits
// (non-negative floats order as unsigned integers), for the FP16 scales:
// over the cells the contraction sums (the box's planes, box may be null),
// the only ones the bank holds.
__global__ void absmax_rows_kernel(const float* __restrict__ w0, const float* __restrict__ bank, int64_t bstride,
                                   int64_t nc, int ns, const int* __restrict__ box, int64_t plane,
                                   unsigned* __restrict__ out) {
  const int row = blockIdx.y;
  const float* src = row == 0 ? w0 : bank + (int64_t)(row - 1) * bstride;
  const CellRange r = box_cells(box, plane, nc);
  float m = 0.0f;
  for (int64_t i = r.lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r.hi;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(__ldg(src + i)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + row, __float_as_uint(m));
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
int64_t umma_cells_per_split(int64_t nc, int ntiles, int sm_count, int ctas_per_sm) {
  const int64_t cap = (int64_t)UM_MAX_GROUPS * UM_GCELLS;
  int64_t splits =
      std::max<int64_t>(1, ((int64_t)ctas_per_sm * sm_count + ntiles - 1) / std::max(ntiles, 1));
  int64_t cps = (nc + splits - 1) / splits;
  cps = std::min(cps, cap);
  cps = (cps + UM_GCELLS - 1) / UM_GCELLS * UM_GCELLS;  // whole groups and staging fills
  return std::max<int64_t>(cps, UM_GCELLS);
}

cudaError_t launch_umma(int tn, int kind, const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns,
                        const int2* rowdesc, int rows, const int2* coldesc, const int4* tiles, const int* collist,
                        int ntc, int ntiles, int splits, const int* box, int64_t plane, unsigned* absmax,
                        double* partials, int* status, cudaStream_t st, size_t min_smem) {
  if (ntc == 0) return cudaSuccess;
  if (kind == UM_FP16) {
    cudaError_t e = cudaMemsetAsync(absmax, 0, (size_t)(ns + 1) * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int64_t per = std::min<int64_t>(1024, std::max<int64_t>(1, (nc + 4095) / 4096));
    absmax_rows_kernel<<<dim3((unsigned)per, (unsigned)(ns + 1)), 256, 0, st>>>(w0, bank, bstride, nc, ns, box, plane,
                                                                                absmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
#define CK_UMMA_CASE(W, K)                                                                                           \
  case W:                                                                                                            \
    return launch_umma_t<W, K>(w0, bank, bstride, nc, ns, rowdesc, rows, coldesc, tiles, collist, ntc, ntiles, splits, \
                               box, plane, absmax, partials, status, st, min_smem);
#define CK_UMMA_KIND(K)        \
  switch (tn) {                \
    CK_UMMA_CASE(32, K)        \
    CK_UMMA_CASE(64, K)        \
    CK_UMMA_CASE(128, K)       \
    CK_UMMA_CASE(160, K)       \
    CK_UMMA_CASE(256, K)       \
    default: return cudaErrorInvalidValue; \
  }
  if (kind == UM_BF16) { CK_UMMA_KIND(UM_BF16) }
  if (kind == UM_FP16) { CK_UMMA_KIND(UM_FP16) }
  CK_UMMA_KIND(UM_TF32)
#undef CK_UMMA_KIND
#undef CK_UMMA_CASE
}

// ---------------------------------------------------------------------------
// Thin tiles (at most kThinOut outputs: few rows or few columns, e.g. the
// 25-row, 5-column tail of order 5 over 16 shells) on the CUDA cores in FP32:
// per MMA such a tile costs the tensor cores as much as a full one.  CTA
// (tile, split) stages the W rows of 256 cells, forms the tile's A_p and B_q
// over them in shared memory and sums A_p B_q for one output per thread (FP32
// over the 256 cells, FP64 across chunks), writing the tcgen05 kernel's
// partials layout, so the same reduction serves both.

constexpr int TH_THREADS = 256;
constexpr int TH_CELLS = 256;
constexpr int TH_PITCH = TH_CELLS + 4;  // 16-byte rows, index 1 mod 8: conflict-free float4 reads across rows

__global__ void __launch_bounds__(TH_THREADS)
    contract_thin_kernel(const float* __restrict__ w0, const float* __restrict__ bank, int64_t bstride, int64_t nc,
                         int ns, int rmax, const int2* __restrict__ rowdesc, int rows, const int2* __restrict__ coldesc,
                         const int4* __restrict__ tiles, const int* __restrict__ collist, int t0, int ntiles, int tn,
                         const int* __restrict__ box, int64_t plane, double* __restrict__ partials) {
  extern __shared__ __align__(16) float th_smem[];
  const int tile_i = t0 + blockIdx.x;
  const int4 tile = tiles[tile_i];
  const int R = rows - tile.x < UM_M ? rows - tile.x : UM_M;  // live rows (<= rmax)
  const int C = tile.w;                                          // live columns (<= kThinMaxCols)
  float* wsb = th_smem;                     // [2][ns + 2][TH_PITCH] W0, W_1 .. W_ns, ones (double-buffered)
  float* As = wsb + 2 * (ns + 2) * TH_PITCH;  // [rmax][TH_PITCH]
  float* Bs = As + rmax * TH_PITCH;         // [kThinMaxCols][TH_PITCH]
  int2* fa = reinterpret_cast<int2*>(Bs + kThinMaxCols * TH_PITCH);  // [rmax] staged rows of W_a, W_b
  int2* fb = fa + rmax;                                                // [kThinMaxCols] staged rows of W_c, W_d
  const int tid = threadIdx.x;
  const int ONE = ns + 1;
  for (int r = tid; r < R; r += TH_THREADS) {  // A_p = W0 W_a W_b, B_q = W_c W_d (an index of -1: the ones row)
    const int2 d = rowdesc[tile.x + r];
    fa[r] = make_int2(d.x >= 0 ? 1 + d.x : ONE, d.y >= 0 ? 1 + d.y : ONE);
  }
  for (int q = tid; q < C; q += TH_THREADS) {
    const int2 d = coldesc[collist[tile.y + q]];
    fb[q] = make_int2(d.x >= 0 ? 1 + d.x : ONE, d.y >= 0 ? 1 + d.y : ONE);
  }
  for (int k = tid; k < 2 * TH_CELLS; k += TH_THREADS) wsb[((k / TH_CELLS) * (ns + 2) + ONE) * TH_PITCH + k % TH_CELLS] = 1.0f;
  int64_t beg, end;  // this split's part of the visited cells (256-cell multiples)
  split_cells(box_cells(box, plane, nc), gridDim.y, TH_CELLS, blockIdx.y, &beg, &end);
  const int o = tid;  // this thread's output: row o / C, column o % C
  const bool live = o < R * C;
  const int orow = live ? o / C : 0, ocol = live ? o % C : 0;
  double dacc = 0.0;
  constexpr int K4 = TH_CELLS / 4;
  // W rows of the chunk at c0 into buffer b: 16-byte asynchronous copies
  // (c0 is a multiple of 256 cells), zero-filled past the end
  auto stage = [&](int64_t c0, int b) {
    const int vc = (int)std::min<int64_t>(TH_CELLS, end - c0);
    float* ws = wsb + b * (ns + 2) * TH_PITCH;
    for (int i = tid; i < (ns + 1) * K4; i += TH_THREADS) {
      const int a = i / K4, k4 = i - a * K4;
      const float* src = (a == 0 ? w0 : bank + (int64_t)(a - 1) * bstride) + c0 + 4 * k4;
      const int n = vc - 4 * k4 >= 4 ? 16 : (vc > 4 * k4 ? 4 * (vc - 4 * k4) : 0);
      cp_async16n(ws + a * TH_PITCH + 4 * k4, n > 0 ? (const void*)src : (const void*)w0, n);
    }
  };
  if (beg < end) stage(beg, 0);
  cp_async_commit();
  int buf = 0;
  for (int64_t c0 = beg; c0 < end; c0 += TH_CELLS, buf ^= 1) {
    if (c0 + TH_CELLS < end) stage(c0 + TH_CELLS, buf ^ 1);  // read two chunks ago, before a barrier
    cp_async_commit();
    cp_async_wait<1>();  // this chunk's copies have landed
    __syncthreads();
    const float* ws = wsb + buf * (ns + 2) * TH_PITCH;
    for (int i = tid; i < (R + C) * K4; i += TH_THREADS) {
      const int r = i / K4, k4 = i - r * K4;
      const bool isa = r < R;
      const int2 f = isa ? fa[r] : fb[r - R];
      const float4 x = *reinterpret_cast<const float4*>(ws + f.x * TH_PITCH + 4 * k4);
      const float4 y = *reinterpret_cast<const float4*>(ws + f.y * TH_PITCH + 4 * k4);
      float4 v = make_float4(x.x * y.x, x.y * y.y, x.z * y.z, x.w * y.w);
      if (isa) {
        const float4 n = *reinterpret_cast<const float4*>(ws + 4 * k4);
        v = make_float4(n.x * v.x, n.y * v.y, n.z * v.z, n.w * v.w);
      }
      *reinterpret_cast<float4*>((isa ? As + r * TH_PITCH : Bs + (r - R) * TH_PITCH) + 4 * k4) = v;
    }
    __syncthreads();
    if (live) {
      const float4* a4 = reinterpret_cast<const float4*>(As + orow * TH_PITCH);
      const float4* b4 = reinterpret_cast<const float4*>(Bs + ocol * TH_PITCH);
      float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll 8
      for (int k = 0; k < K4; k += 2) {
        const float4 x = a4[k], y = b4[k], x1 = a4[k + 1], y1 = b4[k + 1];
        acc0 = fmaf(x.x, y.x, acc0);
        acc0 = fmaf(x.y, y.y, acc0);
        acc0 = fmaf(x.z, y.z, acc0);
        acc0 = fmaf(x.w, y.w, acc0);
        acc1 = fmaf(x1.x, y1.x, acc1);
        acc1 = fmaf(x1.y, y1.y, acc1);
        acc1 = fmaf(x1.z, y1.z, acc1);
        acc1 = fmaf(x1.w, y1.w, acc1);
      }
      dacc += (double)acc0 + (double)acc1;
    }
  }
  cp_async_wait<0>();
  if (live) partials[((int64_t)blockIdx.y * ntiles + tile_i) * (int64_t)(UM_M * tn) + orow * tn + ocol] = dacc;
}

static_assert(kThinMaxOut <= TH_THREADS, "one output per thread");

size_t umma_thin_smem(int ns, int rmax) {
  return (size_t)(2 * (ns + 2) + rmax + kThinMaxCols) * TH_PITCH * sizeof(float) +
         (size_t)(rmax + kThinMaxCols) * sizeof(int2);
}

cudaError_t launch_umma_thin(const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns, int rmax,
                             const int2* rowdesc, int rows, const int2* coldesc, const int4* tiles,
                             const int* collist, int t0, int nthin, int ntiles, int tn, int splits, const int* box,
                             int64_t plane, double* partials, cudaStream_t st) {
  if (nthin == 0) return cudaSuccess;
  const size_t sm = umma_thin_smem(ns, rmax);
  cudaError_t e = cudaFuncSetAttribute(contract_thin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  contract_thin_kernel<<<dim3((unsigned)nthin, (unsigned)splits), TH_THREADS, sm, st>>>(
      w0, bank, bstride, nc, ns, rmax, rowdesc, rows, coldesc, tiles, collist, t0, ntiles, tn, box, plane, partials);
  return cudaGetLastError();
}

cudaError_t launch_umma_reduce(const double* partials, int splits, int ntiles, int tn, const int4* tiles,
                               const int* collist, const int2* rowdesc, int rows, const int2* coldesc, int mask,
                               int ns, const int64_t* bases, double* out, cudaStream_t st) {
  UmmaBases B;
  for (int n = 0; n <= CK_MAX_ORDER; ++n) B.base[n] = bases[n];
  const int64_t total = (int64_t)ntiles * UM_M * tn * 32;  // a warp per partial element
  reduce_umma_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(partials, splits, ntiles, tn, tiles, collist,
                                                                      rowdesc, rows, coldesc, mask, ns, B, out);
  return cudaGetLastError();
}

}  // namespace ck
