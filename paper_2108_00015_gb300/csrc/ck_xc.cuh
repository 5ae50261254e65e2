// ck_xc.cuh -- the last inverse FFT pass fused with the summation stage:
// W_s = N *** K_s (Sec. 2.4) leaves the x transform straight into shared
// memory, where the order-2 and order-3 products of Eq. 11,
//   S2[a]    = sum_r N(r) W_a(r),
//   S3[a][b] = sum_r N(r) W_a(r) W_b(r)   (a <= b kept),
// are accumulated without W_s ever being written to global memory.
//
// Tiles and transforms.  A tile is kRows consecutive grid rows (y, z) of
// every shell; a job fills the kT transform lines with SPJ = kT / kRows
// shells of those rows (line c: row c / SPJ, shell q SPJ + c % SPJ).  The
// half-spectrum rows of a job are staged with cp.async (the next job's
// while the current one is transformed), unpacked into the half-length
// complex sequence and transformed; the last iteration writes the real rows
// into a store that holds the whole tile for every shell.
//
// Sums on the tensor cores.  Over the cells of a tile, S3 and S2 form one
// rank-K update D[a][b] += sum_c A[a][c] B[c][b] with A[a][c] = N(c) W_a(c),
// B[c][b] = W_b(c) for b < NS and B[c][NS..] = 1 (column 16 of the third
// n-tile for NS = 16).  Each warp takes k-steps of 8 cells and issues
// m16n8k8 TF32 MMAs whose fragments come straight from the store: lane
// (g, t) = (lane / 4, lane % 4) loads W_g and W_{g+8} at cells t and t + 4,
// which are both its A elements (times N) and its B elements.  Operands are
// split x = hi + lo into two TF32 numbers and the product is taken as
// hi*hi + hi*lo + lo*hi (three MMAs; the dropped lo*lo term is below
// 2^-22 relative), accumulated in FP32 over a tile, in FP32 over
// kFlushTiles tile sums, then in FP64 registers (FP64 throughput is low).  At the end the warps' FP64 sums are added in a fixed order
// and each CTA writes its partials (reduced across CTAs by the caller).
//
// NS is the shell count rounded up to 2, 4, 8 or 16; shells at or beyond
// `nshells` are staged as zeros and their outputs ignored.
#pragma once

#include "ck_fft_core.cuh"
#include "ck_mma.cuh"

namespace ck {
namespace fft {

constexpr int kWarps = kThreads / 32;
// Tiles whose FP32 sums are added in FP32 before one FP64 flush: the FP64
// pipe is narrow, and (24 + kFlushTiles) FP32 roundings stay below 1e-5.
constexpr int kFlushTiles = 32;

__host__ __device__ constexpr int xc_rows(int NS) { return NS >= kT ? 1 : kT / NS; }  // grid rows per tile
__host__ __device__ constexpr int xc_spj(int NS) { return kT / xc_rows(NS); }         // shells per job
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// The grid rows (y, z) a pass visits: with a support box (the cells where
// W_0 may be nonzero, {x0, x1, y0, y1, z0, z1} inclusive, in device memory)
// the rows with y0 <= y <= y1 and z0 <= z <= z1 in order, since the sums of
// Eq. 11 vanish elsewhere; without one (box null) every row.
struct RowMap {
  int64_t ny, y0, nyb, z0;
  int64_t count;  // rows visited
  __device__ __forceinline__ int64_t row(int64_t c) const { return (z0 + c / nyb) * ny + y0 + c % nyb; }
};

__device__ __forceinline__ RowMap row_map(const int* box, int64_t rows, int ny) {
  if (!box) return RowMap{ny, 0, ny, 0, rows};
  const int y0 = box[2], z0 = box[4];
  const int64_t nyb = box_len(y0, box[3]), nzb = box_len(z0, box[5]);
  return RowMap{ny, y0, nyb > 0 ? nyb : 1, z0, nyb > 0 && nzb > 0 ? nyb * nzb : 0};
}

// Shared-memory layout of the fused kernel (byte offsets).
struct XcLayout {
  size_t s0, s1, u, w, tws, twn, wst, nb0, nb1, total;
  int tcp;  // cells per tile rounded up to the 8-cell k-step
};

__host__ __device__ inline XcLayout xc_layout(int M, int NS, int ntw) {
  const int TC = xc_rows(NS) * 2 * M;
  XcLayout L{};
  L.tcp = (TC + 7) / 8 * 8;
  size_t o = 0;
  L.s0 = o;   o += align16((size_t)kT * stage_pitch(M) * sizeof(float2));
  L.s1 = o;   o += align16((size_t)kT * stage_pitch(M) * sizeof(float2));
  L.u = o;    o += align16((size_t)(M + 1) * kT * sizeof(float2));
  L.w = o;    o += align16((size_t)(M + 1) * kT * sizeof(float2));
  L.tws = o;  o += align16((size_t)ntw * sizeof(float2));
  L.twn = o;  o += align16((size_t)(M + 1) * sizeof(float2));
  L.wst = o;  o += align16((size_t)NS * L.tcp * sizeof(float));
  L.nb0 = o;  o += align16((size_t)L.tcp * sizeof(float));
  L.nb1 = o;  o += align16((size_t)L.tcp * sizeof(float));
  // the final cross-warp sum reuses the buffers from offset 0
  const size_t red = (size_t)kWarps * NS * (NS + 1) * sizeof(double);
  L.total = o > red ? o : red;
  return L;
}

// Per-iteration twiddle entries of the half-length transform.
inline int xc_ntw(int M) {
  const RPlan p = rplan(M);
  return p.nst > 0 ? tw_table_len(p) : 0;
}

template <int MC, int NS>
__global__ void __launch_bounds__(kThreads, 2)
    xc_contract_kernel(const float2* __restrict__ spec, int64_t spec_stride, const float* __restrict__ w0, int nx,
                       int px, int64_t rows, int ny, const int* __restrict__ box, int nshells, FftLen f,
                       const float2* __restrict__ stw, const float2* __restrict__ tw,
                       double* __restrict__ partials) {
  static_assert(NS == 2 || NS == 4 || NS == 8 || NS == 16, "padded shell counts");
  constexpr int ROWS = xc_rows(NS);
  constexpr int SPJ = xc_spj(NS);
  constexpr int NQ = NS / SPJ;                 // jobs per tile
  constexpr int NOUT = NS + NS * (NS + 1) / 2;
  constexpr int NTW = NS > 8 ? 2 : 1;          // n-tiles of W columns; the next one holds the ones column
  extern __shared__ float4 smem4[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
  const int M = MC > 0 ? MC : nx / 2;
  const int NX = 2 * M;
  const int TC = ROWS * NX;
  const int LP = stage_pitch(M);
  const int ntw = MC > 0 ? tw_table_len(rplan(MC)) : tw_len_rt(f);
  const XcLayout lay = xc_layout(M, NS, ntw);
  const int TCP = lay.tcp;
  float2* s0 = reinterpret_cast<float2*>(sm + lay.s0);
  float2* s1 = reinterpret_cast<float2*>(sm + lay.s1);
  float2* u = reinterpret_cast<float2*>(sm + lay.u);
  float2* w = reinterpret_cast<float2*>(sm + lay.w);
  float2* tws = reinterpret_cast<float2*>(sm + lay.tws);
  float2* twn = reinterpret_cast<float2*>(sm + lay.twn);
  float* wst = reinterpret_cast<float*>(sm + lay.wst);
  auto nbuf = [&](int b) { return reinterpret_cast<float*>(sm + (b ? lay.nb1 : lay.nb0)); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;

  for (int i = threadIdx.x; i < ntw; i += kThreads) tws[i] = __ldg(stw + i);
  for (int i = threadIdx.x; i <= M; i += kThreads) twn[i] = __ldg(tw + i);
  // cells TC..TCP-1 of the store and of both N buffers stay zero
  for (int i = threadIdx.x; i < (TCP - TC) * (NS + 2); i += kThreads) {
    const int r = i / (TCP - TC), c = TC + i % (TCP - TC);
    if (r < NS) wst[r * TCP + c] = 0.0f;
    else nbuf(r - NS)[c] = 0.0f;
  }

  const RowMap rm = row_map(box, rows, ny);
  const int64_t ntiles = (rm.count + ROWS - 1) / ROWS;
  const int np = M / 2 + 1;  // 16-byte copies per staged row (X[0..M], see x_c2r_kernel)
  auto stage = [&](float2* s, float* nb, int64_t t, int q) {
    const int64_t r0 = t * ROWS;  // first visited row of the tile
    for (int idx = threadIdx.x; idx < kT * np; idx += kThreads) {
      const int c = idx / np, k = 2 * (idx - c * np);
      const int i = c / SPJ, sh = q * SPJ + c % SPJ;
      const bool ok = r0 + i < rm.count && sh < nshells;
      cp_async16(s + c * LP + k,
                 ok ? (const void*)(spec + sh * spec_stride + rm.row(r0 + i) * px + k) : (const void*)spec, ok);
    }
    if (q == 0) {
      const int vr = (int)(rm.count - r0 < ROWS ? rm.count - r0 : ROWS);  // visited rows of the tile
      const int64_t vc = (int64_t)vr * NX;                                 // valid cells of the tile
      if (NX % 4 == 0) {  // every row starts on a 16-byte boundary of w0
        for (int idx = threadIdx.x; idx < TC / 4; idx += kThreads) {
          const int64_t c4 = 4 * (int64_t)idx;
          const bool ok = c4 < vc;
          const int i = (int)(c4 / NX);
          cp_async16n(nb + c4, ok ? (const void*)(w0 + rm.row(r0 + i) * NX + (c4 - (int64_t)i * NX)) : (const void*)w0,
                      ok ? 16 : 0);
        }
      } else {  // plain loads: the buffer is not read before the next barrier
        for (int c = threadIdx.x; c < TC; c += kThreads) {
          const int i = c / NX;
          nb[c] = c < vc ? __ldg(w0 + rm.row(r0 + i) * NX + (c - i * NX)) : 0.0f;
        }
      }
    }
  };

  float dacc32[NTW + 1][4];  // this tile
  float mid[NTW + 1][4];     // tiles since the last FP64 flush
  double dacc[NTW + 1][4];
#pragma unroll
  for (int j = 0; j <= NTW; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      mid[j][e] = 0.0f;
      dacc[j][e] = 0.0;
    }
  int since = 0;
  // the ones column: B[k][n] = 1 for n = 0 of the last n-tile
  const uint32_t ones = g == 0 ? 0x3f800000u : 0u;

  int64_t t = blockIdx.x;
  if (t < ntiles) {
    stage(s0, nbuf(0), t, 0);
    cp_async_commit();
    int q = 0, it = 0, kt = 0;  // job in tile, job counter, tile counter of this CTA
    while (true) {
      int64_t tn = t;
      int qn = q + 1;
      if (qn == NQ) {
        qn = 0;
        tn = t + gridDim.x;
      }
      const float2* sc = (it & 1) ? s1 : s0;
      if (tn < ntiles) stage((it & 1) ? s0 : s1, nbuf((kt + 1) & 1), tn, qn);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      // unpack: Z[k] = (X[k] + conj X[M-k]) + i w^-k (X[k] - conj X[M-k])
      for (int idx = threadIdx.x; idx < kT * (M / 2 + 1); idx += kThreads) {
        const int c = idx % kT, k = idx / kT;
        const float2 a = sc[c * LP + k], b = sc[c * LP + M - k];
        const float2 ca = cconj(a), cb = cconj(b);
        u[k * kT + c] = cadd(cadd(a, cb), cmul_mi<true>(cmul(cconj(twn[k]), csub(a, cb))));
        if (k != 0 && 2 * k != M)
          u[(M - k) * kT + c] = cadd(cadd(b, ca), cmul_mi<true>(cmul(cconj(twn[M - k]), csub(b, ca))));
      }
      __syncthreads();
      {
        SmemLd ld{u};
        // line pair cp: row (2 cp) / SPJ, shells q SPJ + (2 cp) % SPJ and the next one
        auto st = [&](int m, int cp, float4 v) {
          const int c = 2 * cp;
          float* dst = wst + (size_t)(q * SPJ + c % SPJ) * TCP + (c / SPJ) * NX + 2 * m;
          *reinterpret_cast<float2*>(dst) = lo2(v);
          *reinterpret_cast<float2*>(dst + TCP) = hi2(v);
        };
        transform<MC, true>(w, u, tws, f, ld, st);
      }
      if (q == NQ - 1) {
        // every shell of tile t is in the store: rank-8 updates per k-step
        const float* nb = nbuf(kt & 1);
#pragma unroll
        for (int j = 0; j <= NTW; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) dacc32[j][e] = 0.0f;
#pragma unroll 1
        for (int c0 = 8 * warp; c0 < TCP; c0 += 8 * kWarps) {
          const float n0 = nb[c0 + tq], n1 = nb[c0 + tq + 4];
          float wv[4];  // W_g(t), W_{g+8}(t), W_g(t+4), W_{g+8}(t+4)
          wv[0] = g < NS ? wst[g * TCP + c0 + tq] : 0.0f;
          wv[2] = g < NS ? wst[g * TCP + c0 + tq + 4] : 0.0f;
          wv[1] = NS > 8 ? wst[(g + 8) * TCP + c0 + tq] : 0.0f;
          wv[3] = NS > 8 ? wst[(g + 8) * TCP + c0 + tq + 4] : 0.0f;
          uint32_t ah[4], al[4], bh[4], bl[4];
          tf32_split(n0 * wv[0], ah[0], al[0]);
          tf32_split(n0 * wv[1], ah[1], al[1]);
          tf32_split(n1 * wv[2], ah[2], al[2]);
          tf32_split(n1 * wv[3], ah[3], al[3]);
#pragma unroll
          for (int e = 0; e < 4; ++e) tf32_split(wv[e], bh[e], bl[e]);
          // n-tile 0: b = g (W_g at t, t + 4); n-tile 1: b = 8 + g
          mma_tf32(dacc32[0], ah, bh[0], bh[2]);
          mma_tf32(dacc32[0], ah, bl[0], bl[2]);
          mma_tf32(dacc32[0], al, bh[0], bh[2]);
          if constexpr (NTW == 2) {
            mma_tf32(dacc32[1], ah, bh[1], bh[3]);
            mma_tf32(dacc32[1], ah, bl[1], bl[3]);
            mma_tf32(dacc32[1], al, bh[1], bh[3]);
          }
          mma_tf32(dacc32[NTW], ah, ones, ones);
          mma_tf32(dacc32[NTW], al, ones, ones);
        }
#pragma unroll
        for (int j = 0; j <= NTW; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) mid[j][e] += dacc32[j][e];
        if (++since == kFlushTiles) {
#pragma unroll
          for (int j = 0; j <= NTW; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              dacc[j][e] += (double)mid[j][e];
              mid[j][e] = 0.0f;
            }
          since = 0;
        }
        __syncthreads();  // the store is rewritten by the next tile
        ++kt;
      }
      if (tn >= ntiles) break;
      t = tn;
      q = qn;
      ++it;
    }
  }
  // warp sums -> shared memory (over the staging buffers), then a fixed-order
  // sum over warps: element (a, b) of D, b = NS for the order-2 column
  __syncthreads();
#pragma unroll
  for (int j = 0; j <= NTW; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) dacc[j][e] += (double)mid[j][e];
  constexpr int DC = NS + 1;
  double* red = reinterpret_cast<double*>(sm);  // [kWarps][NS][DC]
#pragma unroll
  for (int j = 0; j <= NTW; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int a = g + ((e & 2) ? 8 : 0);
      const int n = 2 * tq + (e & 1);
      const int b = j < NTW ? (8 * j + n < NS ? 8 * j + n : -1) : (n == 0 ? NS : -1);
      if (a < NS && b >= 0) red[(warp * NS + a) * DC + b] = dacc[j][e];
    }
  __syncthreads();
  for (int o = threadIdx.x; o < NOUT; o += kThreads) {
    int a, b;
    if (o < NS) {
      a = o;
      b = NS;
    } else {
      int r = o - NS;
      a = 0;
      while (r >= NS - a) {
        r -= NS - a;
        ++a;
      }
      b = a + r;
    }
    double s = 0.0;
    for (int wp = 0; wp < kWarps; ++wp) s += red[(wp * NS + a) * DC + b];
    partials[(int64_t)blockIdx.x * NOUT + o] = s;
  }
}

// ---------------------------------------------------------------------------
// Power-of-two half-lengths M = P Q (P, Q in {4, 8, 16}): the same pass with
// the transform held in registers.  With k = Q k1 + k2 and m = m1 + P m2,
//   z[m1 + P m2] = sum_k2 e^{2 pi i k2 m2 / Q} e^{2 pi i k2 m1 / M}
//                  sum_k1 e^{2 pi i k1 m1 / P} Z[Q k1 + k2],
// so step A (one thread per line and k2) unpacks its P values of Z straight
// from the staged rows, runs a P-point DFT and applies the twiddles; the
// results go through a padded shared transpose T; step B (one thread per
// line and m1) runs the Q-point DFT and writes the real row
// x[2m] = Re z[m], x[2m+1] = Im z[m] into the store W, which takes the
// place of the tile's staged rows (consumed by step A).  A tile is
// LT = 256 / max(P, Q) lines: ROWS = LT / NS grid rows of every shell, all
// transformed at once; one block barrier per tile (two when P != Q or
// ROWS > 1), before the sums.  Warp 0 stages the next tile into the other
// buffer once every warp has arrived on that buffer's "empty" mbarrier
// after the previous tile's sums (the other warps do not wait), with bulk
// asynchronous copies, one per padded half-spectrum row (px = M + 4 complex
// values) and one for the tile's N cells, completing on the buffer's "full"
// mbarrier.  Waits are bounded; a failed wait in any warp ends every warp
// at the next block barrier.
//
// In the sums, k-slot t of a k-step holds cell c0 + 2t and slot t + 4 cell
// c0 + 2t + 1, so that each lane reads its two cells with one 8-byte load.

template <int P, int Q, int NS>
struct XcrShape {
  static constexpr int M = P * Q;
  static constexpr int NX = 2 * M;
  static constexpr int LT = kThreads / (P > Q ? P : Q);  // lines per tile
  static constexpr int ROWS = LT / NS;                   // grid rows per tile
  static constexpr int TC = ROWS * NX;                   // cells per tile
  static constexpr int LP = M + 4;                       // staged row pitch (float2): the padded row, px
  static constexpr int TP = Q * (P + 1);                 // transpose float2 per line
  static constexpr int WP = TC + 8;                      // store pitch per shell (floats), 8 mod 32
  static constexpr size_t s_bytes = align16((size_t)LT * LP * sizeof(float2));
  static constexpr size_t twu_off = 2 * s_bytes;  // e^{+2 pi i k / NX}, k <= M
  static constexpr size_t twq_off = twu_off + align16((size_t)(M + 1) * sizeof(float2));  // [k2][m1], row pitch P + 1: e^{2 pi i k2 m1 / M}
  static constexpr size_t t_off = twq_off + align16((size_t)Q * (P + 1) * sizeof(float2));
  static constexpr size_t nb_off = t_off + align16((size_t)LT * TP * sizeof(float2));
  static constexpr size_t nb_bytes = align16((size_t)TC * sizeof(float));
  static constexpr size_t bar_off = nb_off + 2 * nb_bytes;
  static constexpr size_t red_bytes = (size_t)kWarps * NS * (NS + 1) * sizeof(double);
  static constexpr size_t total0 = bar_off + 32;  // full[2], empty[2]
  static constexpr size_t total = total0 > red_bytes ? total0 : red_bytes;
  static_assert(ROWS >= 1 && LT % NS == 0, "a tile holds whole rows of every shell");
  static_assert((size_t)NS * WP * sizeof(float) <= s_bytes, "the store fits in a staging buffer");
  // steps A and B of a line in one warp, and W[line] over the line's staged row
  static constexpr bool kWarpLocal = P == Q && ROWS == 1 && WP * sizeof(float) == LP * sizeof(float2);
  static_assert(TC % 32 == 0, "whole k-steps per tile and a conflict-free store pitch");
  static_assert((LP * sizeof(float2)) % 16 == 0 && (NX * sizeof(float)) % 16 == 0, "16-byte bulk copies");
  static_assert(red_bytes <= bar_off, "the final sum does not reach the barriers");
};


template <int P, int Q, int NS>
__global__ void __launch_bounds__(kThreads, 2)
    xcr_contract_kernel(const float2* __restrict__ spec, int64_t spec_stride, const float* __restrict__ w0, int px,
                        int64_t rows, int ny, const int* __restrict__ box, int nshells, const float2* __restrict__ tw,
                        double* __restrict__ partials, int* status) {
  using S = XcrShape<P, Q, NS>;
  constexpr int M = S::M, NX = S::NX, LT = S::LT, ROWS = S::ROWS, TC = S::TC, LP = S::LP, TP = S::TP, WP = S::WP;
  constexpr int NOUT = NS + NS * (NS + 1) / 2;
  constexpr int NTW = NS > 8 ? 2 : 1;
  extern __shared__ float4 smem4[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
  // staging buffer b at b * s_bytes, N buffer b at nb_off + b * nb_bytes
  auto sbuf = [&](int b) { return reinterpret_cast<float2*>(sm + b * S::s_bytes); };
  auto nbuf = [&](int b) { return reinterpret_cast<float*>(sm + S::nb_off + b * S::nb_bytes); };
  float2* twu = reinterpret_cast<float2*>(sm + S::twu_off);
  float2* twq = reinterpret_cast<float2*>(sm + S::twq_off);
  float2* T = reinterpret_cast<float2*>(sm + S::t_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + S::bar_off);  // [2] a tile staged (bulk-copy bytes)
  uint64_t* empty = full + 2;                                       // [2] every warp's sums of the buffer done
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int nsv = nshells < NS ? nshells : NS;  // shells with data; the other lines stay zero

  // tw[t] = e^{-2 pi i t / NX}, t < NX
  for (int i = tid; i <= M; i += kThreads) twu[i] = cconj(__ldg(tw + i));
  for (int i = tid; i < M; i += kThreads) twq[(i / P) * (P + 1) + i % P] = cconj(__ldg(tw + 2 * ((i / P) * (i % P))));
  for (int i = tid; i < (int)(2 * S::s_bytes / 16); i += kThreads) reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], kWarps);
    mbar_init(&empty[1], kWarps);
  }
  fence_async_shared();  // zeroed buffers and barrier initialisation before any bulk copy
  __syncthreads();

  const RowMap rm = row_map(box, rows, ny);
  const int64_t ntiles = (rm.count + ROWS - 1) / ROWS;
  // the 8-cell k-steps of a row that can meet a nonzero N: those overlapping
  // the box's cells x0 .. x1 (W_0 = N vanishes outside them, and so do the
  // terms of both sums)
  static_assert(NX % 8 == 0, "whole k-steps per grid row");
  int kx0 = 0, nks = NX / 8;
  if (box && box[0] <= box[1]) {
    kx0 = max(box[0], 0) / 8;
    nks = max(0, min(NX, box[1] + 8) / 8 - kx0);
  }
  // thread 0: bulk copies of tile t into staging buffer b and N buffer nbi
  // warp 0: lane 0 arms the barrier, then the lanes issue one copy each
  // (a spectrum row per shell and visited row, and the row's N cells)
  auto stage = [&](int b, int nbi, int64_t t) {
    const int64_t r0 = t * ROWS;  // first visited row of the tile
    const int vr = (int)(rm.count - r0 < ROWS ? rm.count - r0 : ROWS);
    const uint32_t row_bytes = LP * sizeof(float2);
    if (lane == 0)
      mbar_arrive_expect_tx(&full[b], (uint32_t)(nsv * vr) * row_bytes + (uint32_t)(vr * NX * sizeof(float)));
    __syncwarp();
    const int nrows = nsv * vr;
    for (int j = lane; j < nrows + vr; j += 32) {
      if (j < nrows) {
        const int sh = j / vr, i = j - sh * vr;
        bulk_g2s(sbuf(b) + (sh * ROWS + i) * LP, spec + sh * spec_stride + rm.row(r0 + i) * px, row_bytes, &full[b]);
      } else {
        const int i = j - nrows;
        bulk_g2s(nbuf(nbi) + i * NX, w0 + rm.row(r0 + i) * NX, (uint32_t)(NX * sizeof(float)), &full[b]);
      }
    }
  };

  float dacc32[NTW + 1][4];  // this tile: hi * hi
  float dsm32[NTW + 1][4];   // this tile: hi * lo + lo * hi (a second chain of MMAs)
  float mid[NTW + 1][4];     // tiles since the last FP64 flush
  double dacc[NTW + 1][4];
#pragma unroll
  for (int j = 0; j <= NTW; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      mid[j][e] = 0.0f;
      dacc[j][e] = 0.0;
    }
  const uint32_t ones = g == 0 ? 0x3f800000u : 0u;
  int since = 0;

  int64_t t = blockIdx.x;
  int issued = 0, used = 0;  // tiles staged / consumed by this CTA
  if (t < ntiles && warp == 0) stage(0, 0, t);
  if (t < ntiles) issued = 1;
  for (int kt = 0; t < ntiles; t += gridDim.x, ++kt) {
    const int64_t tn = t + gridDim.x;
    bool ok = mbar_wait(&full[kt & 1], (uint32_t)(kt >> 1) & 1u, status);
    if (ok) used = kt + 1;
    // the next tile goes to the buffers of tile kt - 1 once every warp has
    // finished that tile's sums (empty barrier); the other warps go on
    if (warp == 0 && ok && tn < ntiles) {
      if (kt >= 1) ok = mbar_wait(&empty[(kt + 1) & 1], (uint32_t)((kt - 1) >> 1) & 1u, status);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (ok) {
        stage((kt + 1) & 1, (kt + 1) & 1, tn);
        issued = kt + 2;
      }
    }
    float* W = reinterpret_cast<float*>(sbuf(kt & 1));
    const int64_t r0 = t * ROWS;
    const int vc = (int)(rm.count - r0 < ROWS ? rm.count - r0 : ROWS) * NX;  // cells of the tile with data
    // step A: unpack Z[Q k1 + k2] = (X[k] + conj X[M-k]) + i e^{2 pi i k/NX} (X[k] - conj X[M-k]),
    // P-point inverse DFT over k1, twiddle e^{2 pi i k2 m1 / M}, into T
    if (ok && tid < LT * Q) {
      const int l = tid / Q, k2 = tid - l * Q;
      const float2* xr = sbuf(kt & 1) + l * LP;
      float2 v[P];
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) {
        const int k = Q * k1 + k2;
        const float2 a = xr[k], cb = cconj(xr[M - k]);
        v[k1] = cadd(cadd(a, cb), cmul_mi<true>(cmul(twu[k], csub(a, cb))));
      }
      dft<P, true>(v);
      float2* tr = T + l * TP + k2 * (P + 1);
      const float2* tk = twq + k2 * (P + 1);
      tr[0] = v[0];
#pragma unroll
      for (int m1 = 1; m1 < P; ++m1) tr[m1] = cmul(v[m1], tk[m1]);
    }
    // T complete, staged rows consumed.  With P == Q and one grid row per
    // tile, the threads of a line in steps A and B are the same warp's, and
    // the store row W[shell] covers exactly the bytes of that line's staged
    // row: the warp alone touches them, so it need not wait for the others.
    if constexpr (S::kWarpLocal) __syncwarp();
    else if (__syncthreads_or(!ok)) break;
    // step B: Q-point inverse DFT over k2 of column m1
    const int lb = tid / P, m1 = tid - lb * P;
    if (ok && tid < LT * P) {
      float2 z[Q];
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) z[k2] = T[lb * TP + k2 * (P + 1) + m1];
      dft<Q, true>(z);
      const int sh = lb / ROWS, i = lb - sh * ROWS;
      float* wr = W + sh * WP + i * NX + 2 * m1;
#pragma unroll
      for (int m2 = 0; m2 < Q; ++m2) *reinterpret_cast<float2*>(wr + 2 * P * m2) = z[m2];
    }
    // the store complete everywhere; a failed wait anywhere ends every warp here
    if (__syncthreads_or(!ok)) break;
    // rank-8 updates on the tensor cores (see xc_contract_kernel)
    {
      const float* nb = nbuf(kt & 1);
#pragma unroll
      for (int j = 0; j <= NTW; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          dacc32[j][e] = 0.0f;
          dsm32[j][e] = 0.0f;
        }
#pragma unroll 2
      for (int q = warp; q < ROWS * nks; q += kWarps) {
        const int c0 = ROWS == 1 ? 8 * (kx0 + q) : (q / nks) * NX + 8 * (kx0 + q % nks);
        const int c = c0 + 2 * tq;
        float2 nn = *reinterpret_cast<const float2*>(nb + c);
        if (c >= vc) nn = make_float2(0.f, 0.f);  // rows past the grid (last tile)
        const float2 wa = g < NS ? *reinterpret_cast<const float2*>(W + g * WP + c) : make_float2(0.f, 0.f);
        const float2 wb = NS > 8 ? *reinterpret_cast<const float2*>(W + (g + 8) * WP + c) : make_float2(0.f, 0.f);
        const float av[4] = {nn.x * wa.x, nn.x * wb.x, nn.y * wa.y, nn.y * wb.y};
        const float bv[4] = {wa.x, wa.y, wb.x, wb.y};
        uint32_t ah[4], al[4], bh[4], bl[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ah[e] = tf32_trunc(av[e]);
          al[e] = __float_as_uint(av[e] - __uint_as_float(ah[e]));
          bh[e] = tf32_trunc(bv[e]);
          bl[e] = __float_as_uint(bv[e] - __uint_as_float(bh[e]));
        }
        // n-tile 0: B[k][g] = W_g; n-tile 1: B[k][g] = W_{g+8}; last: ones column
        mma_tf32(dacc32[0], ah, bh[0], bh[1]);
        mma_tf32(dsm32[0], ah, bl[0], bl[1]);
        mma_tf32(dsm32[0], al, bh[0], bh[1]);
        if constexpr (NTW == 2) {
          mma_tf32(dacc32[1], ah, bh[2], bh[3]);
          mma_tf32(dsm32[1], ah, bl[2], bl[3]);
          mma_tf32(dsm32[1], al, bh[2], bh[3]);
        }
        mma_tf32(dacc32[NTW], ah, ones, ones);
        mma_tf32(dsm32[NTW], al, ones, ones);
      }
#pragma unroll
      for (int j = 0; j <= NTW; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) mid[j][e] += dacc32[j][e] + dsm32[j][e];
      if (++since == kFlushTiles) {
#pragma unroll
        for (int j = 0; j <= NTW; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            dacc[j][e] += (double)mid[j][e];
            mid[j][e] = 0.0f;
          }
        since = 0;
      }
    }
    // this warp is done with the tile's buffers; the next tile's step A
    // writes T only after this tile's second barrier
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[kt & 1]);
  }
  // after a timed-out wait: let the copies already issued land (bounded)
  if (tid == 0)
    for (int k = used; k < issued; ++k)
      if (!mbar_wait(&full[k & 1], (uint32_t)(k >> 1) & 1u, status)) break;
  __syncthreads();
#pragma unroll
  for (int j = 0; j <= NTW; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) dacc[j][e] += (double)mid[j][e];
  constexpr int DC = NS + 1;
  double* red = reinterpret_cast<double*>(sm);  // [kWarps][NS][DC]
#pragma unroll
  for (int j = 0; j <= NTW; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int a = g + ((e & 2) ? 8 : 0);
      const int n = 2 * tq + (e & 1);
      const int b = j < NTW ? (8 * j + n < NS ? 8 * j + n : -1) : (n == 0 ? NS : -1);
      if (a < NS && b >= 0) red[(warp * NS + a) * DC + b] = dacc[j][e];
    }
  __syncthreads();
  for (int o = tid; o < NOUT; o += kThreads) {
    int a, b;
    if (o < NS) {
      a = o;
      b = NS;
    } else {
      int r = o - NS;
      a = 0;
      while (r >= NS - a) {
        r -= NS - a;
        ++a;
      }
      b = a + r;
    }
    double s = 0.0;
    for (int wp = 0; wp < kWarps; ++wp) s += red[(wp * NS + a) * DC + b];
    partials[(int64_t)blockIdx.x * NOUT + o] = s;
  }
}

}  // namespace fft
}  // namespace ck
