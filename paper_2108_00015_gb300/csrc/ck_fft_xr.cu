// ck_fft_xr.cu -- the x passes of 512-cell rows with the transforms in
// registers: real rows of the field -> half-spectrum rows (the first pass of
// the forward transform of Sec. 2.4's convolution) and back (the last pass
// of the inverse, where the plan keeps the bank).
//
// A row of NX = 512 reals is z[n] = x[2n] + i x[2n+1], n < M = 256.  With
// n = 16 n1 + n2 and k = k1 + 16 k2,
//   Z[k1 + 16 k2] = sum_n2 w16^(n2 k2) w256^(n2 k1) sum_n1 w16^(n1 k1) z[16 n1 + n2]
// (w_N = e^{-2 pi i / N}).  Step A: thread (row, n2) runs the 16-point DFT
// over n1 and applies w256^(n2 k1) into a padded transpose T.  Step B:
// thread (row, k1) runs the 16-point DFT over n2 and writes Z over the row's
// staged reals.  Then X[k] = E[k] + e^{-2 pi i k / NX} O[k] with
// E = (Z[k] + conj Z[M-k]) / 2 and O = (Z[k] - conj Z[M-k]) / 2i, k = 0..M,
// goes to the half-spectrum row, zeros in its padding columns.
//
// A tile is 16 rows; warp w owns rows 2w and 2w + 1 end to end (its own
// cp.async staging, double-buffered, its own part of T), so no step waits
// for another warp.  With a support box only the box's rows are visited
// (the field vanishes on the others, which are not written).
#include <algorithm>

#include "ck_fft_core.cuh"

namespace ck {
namespace fft {

namespace {

constexpr int XR_M = 256, XR_NX = 512, XR_P = 16;
constexpr int XR_ROWS = 16;                         // rows per tile
constexpr int XR_TP = XR_P * (XR_P + 1);            // float2 per row of T (pitch P + 1)
constexpr size_t XR_ROW_BYTES = XR_NX * sizeof(float);
constexpr size_t XR_STAGE = (size_t)XR_ROWS * XR_ROW_BYTES;            // one buffer of staged rows
constexpr size_t XR_T_OFF = 2 * XR_STAGE;
constexpr size_t XR_TWQ_OFF = XR_T_OFF + (size_t)XR_ROWS * XR_TP * sizeof(float2);
constexpr size_t XR_TWN_OFF = XR_TWQ_OFF + (size_t)XR_TP * sizeof(float2);
constexpr size_t XR_SMEM = XR_TWN_OFF + (size_t)(XR_M + 1) * sizeof(float2);
static_assert(kThreads == 2 * XR_P * (kThreads / 32) && XR_ROWS == 2 * (kThreads / 32), "two rows per warp");

__global__ void __launch_bounds__(kThreads, 2)
    xr2c_reg_kernel(const float* __restrict__ in, float2* __restrict__ out, int px, int64_t rows,
                    const float2* __restrict__ tw, const int* __restrict__ box, int ny) {
  extern __shared__ float4 smem4[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
  float2* T = reinterpret_cast<float2*>(sm + XR_T_OFF);
  float2* twq = reinterpret_cast<float2*>(sm + XR_TWQ_OFF);  // [n2][k1]: w256^(n2 k1)
  float2* twn = reinterpret_cast<float2*>(sm + XR_TWN_OFF);  // [k]: e^{-2 pi i k / NX}, k <= M
  for (int i = threadIdx.x; i < XR_P * XR_P; i += kThreads)
    twq[(i / XR_P) * (XR_P + 1) + i % XR_P] = __ldg(tw + 2 * ((i / XR_P) * (i % XR_P)));
  for (int i = threadIdx.x; i <= XR_M; i += kThreads) twn[i] = __ldg(tw + i);
  __syncthreads();  // the tables, before any warp uses them

  // visited rows: every row, or the box's (y0..y1, z0..z1) in order
  int64_t y0 = 0, nyb = ny > 0 ? ny : 1, z0 = 0, count = rows;
  if (box) {
    y0 = box[2];
    nyb = box_len(box[2], box[3]);
    z0 = box[4];
    const int64_t nzb = box_len(box[4], box[5]);
    count = nyb > 0 && nzb > 0 ? nyb * nzb : 0;
    if (nyb <= 0) nyb = 1;
  }
  auto row_of = [=](int64_t c) { return box ? (z0 + c / nyb) * ny + y0 + c % nyb : c; };
  const int64_t ntiles = (count + XR_ROWS - 1) / XR_ROWS;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane >> 4, j = lane & 15;  // this lane's row of the warp's two, index in the row
  const int r = 2 * warp + half;              // row of the tile
  auto stage = [&](int b, int64_t t) {
    // the warp's two rows: 2 x 128 pieces of 16 bytes, 8 per lane
    float* dst = reinterpret_cast<float*>(sm + b * XR_STAGE);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int piece = lane + 32 * q;  // 0..255
      const int rr = 2 * warp + (piece >> 7), off = (piece & 127) * 4;
      const int64_t c = t * XR_ROWS + rr;
      const bool ok = c < count;
      cp_async16(dst + rr * XR_NX + off, ok ? in + row_of(c) * XR_NX + off : in, ok);
    }
  };
  int64_t t = blockIdx.x;
  if (t < ntiles) stage(0, t);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) stage((it + 1) & 1, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // the warp's rows of tile t are staged
    float2* zr = reinterpret_cast<float2*>(sm + (it & 1) * XR_STAGE) + r * XR_M;  // z[n] of row r
    float2* tr = T + r * XR_TP;
    // step A: thread (r, n2 = j)
    {
      float2 v[XR_P];
#pragma unroll
      for (int n1 = 0; n1 < XR_P; ++n1) v[n1] = zr[XR_P * n1 + j];
      dft<XR_P, false>(v);
      const float2* tk = twq + j * (XR_P + 1);
      tr[j * (XR_P + 1)] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < XR_P; ++k1) tr[j * (XR_P + 1) + k1] = cmul(v[k1], tk[k1]);
    }
    __syncwarp();  // T of the warp's rows complete; their staged reals read
    // step B: thread (r, k1 = j): Z[j + 16 k2] over the staged row
    {
      float2 y[XR_P];
#pragma unroll
      for (int n2 = 0; n2 < XR_P; ++n2) y[n2] = tr[n2 * (XR_P + 1) + j];
      dft<XR_P, false>(y);
#pragma unroll
      for (int k2 = 0; k2 < XR_P; ++k2) zr[j + XR_P * k2] = y[k2];
    }
    __syncwarp();  // Z of the warp's rows complete
    // the even / odd split into the half-spectrum row (and its padding)
    const int64_t c = t * XR_ROWS + r;
    if (c < count) {
      float2* orow = out + row_of(c) * px;
      for (int k = j; k < px; k += XR_P) {
        float2 X = make_float2(0.f, 0.f);
        if (k <= XR_M) {
          const float2 zk = zr[k == XR_M ? 0 : k];
          const float2 zc = cconj(zr[k == 0 ? 0 : XR_M - k]);
          const float2 E = cscale(cadd(zk, zc), 0.5f);
          const float2 O = cscale(cmul_mi<false>(csub(zk, zc)), 0.5f);
          X = cadd(E, cmul(twn[k], O));
        }
        orow[k] = X;
      }
    }
    __syncwarp();  // Z read before the buffer is staged again
  }
  cp_async_wait<0>();
}

// The inverse x pass of 512-cell rows: half-spectrum rows X[0..M] (pitch
// px) -> real rows, z = IDFT_M(Z) (unnormalised) with
// Z[k] = (X[k] + conj X[M-k]) + i e^{2 pi i k / NX} (X[k] - conj X[M-k]), and
// x[2m] = Re z[m], x[2m+1] = Im z[m].  Step A unpacks and runs the inverse
// 16-point DFT over k1 (k = 16 k1 + k2), step B the one over k2, writing
// z[m1 + 16 m2] straight to the output row.  Rows are visited as in
// x_c2r_kernel: every row, or the rows of the box's planes of every shell;
// visited row r is in + row(r) px and goes to out + shell * out_shell_stride
// + (row in the shell) * NX.
constexpr int XC_LP = XR_M + 4;  // staged row pitch (float2): X[0..M] and padding
constexpr size_t XC_STAGE = (size_t)XR_ROWS * XC_LP * sizeof(float2);
constexpr size_t XC_T_OFF = 2 * XC_STAGE;
constexpr size_t XC_TWQ_OFF = XC_T_OFF + (size_t)XR_ROWS * XR_TP * sizeof(float2);
constexpr size_t XC_TWU_OFF = XC_TWQ_OFF + (size_t)XR_TP * sizeof(float2);
constexpr size_t XC_SMEM = XC_TWU_OFF + (size_t)(XR_M + 1) * sizeof(float2);

__global__ void __launch_bounds__(kThreads, 2)
    xc2r_reg_kernel(const float2* __restrict__ in, float* __restrict__ out, int px, int64_t rows,
                    int64_t rows_per_shell, int64_t out_shell_stride, const float2* __restrict__ tw,
                    const int* __restrict__ box, int ny) {
  extern __shared__ float4 smem4[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
  float2* T = reinterpret_cast<float2*>(sm + XC_T_OFF);
  float2* twq = reinterpret_cast<float2*>(sm + XC_TWQ_OFF);  // [k2][m1]: e^{+2 pi i k2 m1 / M}
  float2* twu = reinterpret_cast<float2*>(sm + XC_TWU_OFF);  // [k]: e^{+2 pi i k / NX}, k <= M
  for (int i = threadIdx.x; i < XR_P * XR_P; i += kThreads)
    twq[(i / XR_P) * (XR_P + 1) + i % XR_P] = cconj(__ldg(tw + 2 * ((i / XR_P) * (i % XR_P))));
  for (int i = threadIdx.x; i <= XR_M; i += kThreads) twu[i] = cconj(__ldg(tw + i));
  __syncthreads();  // the tables, before any warp uses them

  // visited rows: every row, or the rows of the planes box[4] .. box[5] of
  // every shell, numbered q = shell * nrb + row in those planes
  int64_t count = rows, nrb = rows_per_shell, rb0 = 0;
  if (box) {
    nrb = (int64_t)box_len(box[4], box[5]) * ny;
    rb0 = (int64_t)box[4] * ny;
    count = (rows / rows_per_shell) * nrb;
  }
  auto row_of = [&](int64_t q) -> int64_t {  // the row's index in [shell][rows_per_shell]
    if (!box) return q;
    const int64_t sh = q / nrb;
    return sh * rows_per_shell + rb0 + (q - sh * nrb);
  };
  const int64_t ntiles = (count + XR_ROWS - 1) / XR_ROWS;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane >> 4, j = lane & 15;
  const int r = 2 * warp + half;
  constexpr int NPC = XC_LP * (int)sizeof(float2) / 16;  // 16-byte pieces per staged row (px = XC_LP)
  auto stage = [&](int b, int64_t t) {
    float2* dst = reinterpret_cast<float2*>(sm + b * XC_STAGE);
    for (int piece = lane; piece < 2 * NPC; piece += 32) {
      const int rr = 2 * warp + piece / NPC, off = 2 * (piece % NPC);
      const int64_t c = t * XR_ROWS + rr;
      const bool ok = c < count;
      cp_async16(dst + rr * XC_LP + off, ok ? (const void*)(in + row_of(c) * px + off) : (const void*)in, ok);
    }
  };
  int64_t t = blockIdx.x;
  if (t < ntiles) stage(0, t);
  cp_async_commit();
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) stage((it + 1) & 1, tn);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();  // the warp's rows of tile t are staged
    const float2* xr = reinterpret_cast<const float2*>(sm + (it & 1) * XC_STAGE) + r * XC_LP;
    float2* tr = T + r * XR_TP;
    // step A: thread (r, k2 = j): unpack Z[16 k1 + k2], inverse DFT over k1, twiddle
    {
      float2 v[XR_P];
#pragma unroll
      for (int k1 = 0; k1 < XR_P; ++k1) {
        const int k = XR_P * k1 + j;
        const float2 a = xr[k], cb = cconj(xr[XR_M - k]);
        v[k1] = cadd(cadd(a, cb), cmul_mi<true>(cmul(twu[k], csub(a, cb))));
      }
      dft<XR_P, true>(v);
      const float2* tk = twq + j * (XR_P + 1);
      tr[j * (XR_P + 1)] = v[0];
#pragma unroll
      for (int m1 = 1; m1 < XR_P; ++m1) tr[j * (XR_P + 1) + m1] = cmul(v[m1], tk[m1]);
    }
    __syncwarp();  // T of the warp's rows complete
    // step B: thread (r, m1 = j): z[m1 + 16 m2] -> cells 2 (m1 + 16 m2), + 1
    const int64_t c = t * XR_ROWS + r;
    {
      float2 z[XR_P];
#pragma unroll
      for (int k2 = 0; k2 < XR_P; ++k2) z[k2] = tr[k2 * (XR_P + 1) + j];
      dft<XR_P, true>(z);
      if (c < count) {
        const int64_t row = row_of(c), sh = row / rows_per_shell, rr = row - sh * rows_per_shell;
        float* orow = out + sh * out_shell_stride + rr * XR_NX + 2 * j;
#pragma unroll
        for (int m2 = 0; m2 < XR_P; ++m2) *reinterpret_cast<float2*>(orow + 2 * XR_P * m2) = z[m2];
      }
    }
    __syncwarp();  // T and the staged rows read before they are written again
  }
  cp_async_wait<0>();
}

}  // namespace

void launch_xc2r_reg(const float2* in, float* out, int px, int64_t rows, int64_t rows_per_shell,
                     int64_t out_shell_stride, const float2* tw, int sm_count, cudaStream_t st, const int* box,
                     int ny) {
  const int64_t ntiles = (rows + XR_ROWS - 1) / XR_ROWS;  // the grid covers every row; a box visits fewer
  allow_smem(xc2r_reg_kernel, XC_SMEM);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)2 * sm_count));
  xc2r_reg_kernel<<<grid, kThreads, XC_SMEM, st>>>(in, out, px, rows, rows_per_shell, out_shell_stride, tw, box,
                                                   ny);
}

void launch_xr2c_reg(const float* in, float2* out, int px, int64_t rows, const float2* tw, int sm_count,
                     cudaStream_t st, const int* box, int ny) {
  const int64_t ntiles = (rows + XR_ROWS - 1) / XR_ROWS;  // the grid covers every row; a box visits fewer
  allow_smem(xr2c_reg_kernel, XR_SMEM);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)2 * sm_count));
  xr2c_reg_kernel<<<grid, kThreads, XR_SMEM, st>>>(in, out, px, rows, tw, box, ny);
}

}  // namespace fft
}  // namespace ck
