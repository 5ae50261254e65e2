// ck_zconv.cu -- the z step of the convolution stage (Sec. 2.4, Eqs. 9-10)
// done directly along z, in place of the forward and inverse z transforms.
//
// A shell reaches at most m_s planes in z (|m_z| <= m_s for its offsets,
// Sec. 2.3), so once the field has been transformed along x and y, the
// convolution along z of one column (kx, ky) is a short even filter:
//   W_s(kx, ky, z) = sum_{|d| <= m_s} K_s^xy(kx, ky, |d|) D(kx, ky, (z - d) mod n_z),
// K_s^xy(., ., d) the (x, y) transform of the plane m_z = d of K_s, which is
// real (K_s is even in x and y).  The transform route gives the same
// circular convolution: K^_s(k) = sum_d K_s^xy(d) e^{-2 pi i k_z d / n_z},
// and the unnormalised inverse z transform of K^_s D^ / N_c is
// n_z / N_c sum_d K_s^xy(d) D(z - d).  The table therefore holds
// K_s^xy / (n_x n_y), in groups of 4 shells, with the d = 0 entry halved so
// that every tap multiplies the pair D(z - d) + D(z + d):
//   table[g][kyf][kx][d][j] (kyf = min(ky, n_y - ky): K_s is even in ky;
//   kx < px, zeros for kx > n_x / 2; d < dz, zeros beyond m_s).
//
// Work unit: 32 adjacent columns of a plane (the flattened (ky, kx) index)
// x up to zc output planes of the support box.  The staged planes E (the
// unit's planes plus dz on either side, zeros outside the box) serve every
// shell group; a thread keeps 4 shells x 4 consecutive planes of one
// column in registers and walks the staged column down and up from them,
// one tap at a time, with packed FP32x2 adds and FMAs (a complex value is
// one register pair).  Groups of 4 shells' taps are double-buffered through
// shared memory.
#include <algorithm>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {

namespace {

constexpr int ZC_C = 32;    // columns per unit
constexpr int ZC_NT = 256;  // threads per CTA
constexpr int ZC_R = 4;     // consecutive planes per thread
constexpr int ZC_G = kZconvGroup;  // shells per group
static_assert(ZC_G % 4 == 0, "a group's taps of one plane offset are whole 16-byte pieces");
constexpr int ZC_EP = 34;   // float2 per staged plane (32 columns + 2: conflict-free 8-byte loads)
constexpr int ZC_PASS = (ZC_NT / ZC_C) * ZC_R;  // planes per pass of the CTA
constexpr int ZC_CTAS = 3;  // CTAs per SM
constexpr size_t ZC_SMEM_CAP = 74 * 1024;      // three CTAs per SM

struct ZconvArgs {
  const float2* spec;     // [n_z][n_y][px], transformed along x and y
  float2* out;            // shell s - shell0 at out + (s - shell0) * out_stride
  int64_t out_stride;
  const float* table;     // [group][kyf][px][dz][8]
  int64_t group_stride;   // floats per group
  int64_t plane;          // complex elements per plane: n_y px (the flattened columns)
  const int* in_box;      // box (device) whose planes z = [4] .. [5] hold the field, or null: every plane
  const int* out_box;     // box (device) whose planes are written, or null: every plane
  int px, ny, nz;
  int dz;                 // taps stored per column, a multiple of 4
  int zc;                 // most output planes per unit (shared memory), a multiple of 4
  int shell0, nshells;    // shells written
  int g0, g1;             // groups g0 .. g1 - 1
  int taps[CK_MAX_SHELLS / ZC_G];  // taps used per group (multiple of 4, <= dz)
};

size_t zconv_smem(int dz, int zc) {
  const size_t kp = (size_t)dz * ZC_G + 4;
  return (size_t)(zc + 2 * dz) * ZC_EP * sizeof(float2) + 2 * ZC_C * kp * sizeof(float);
}

// Taps d = 0 .. T - 1 of one pass: acc[j][r] += k_j(d) (E[z - d] + E[z + d])
// for the planes z = qb + r of a column, e pointing at E's row of plane qb
// and kc at the column's taps.  T is a compile-time count, so the loop
// unrolls: each staged row is loaded once, every shared-memory offset is an
// immediate, and the adds and FMAs are packed FP32x2 operations on the
// complex values (each lane rounded as fmaf).
template <int T>
__device__ __forceinline__ void zconv_taps(const float2* e, const float* kc, float2 (&acc)[ZC_G][ZC_R]) {
#pragma unroll
  for (int d = 0; d < T; ++d) {
    const float4 kq = *reinterpret_cast<const float4*>(kc + d * ZC_G);
    const float k[ZC_G] = {kq.x, kq.y, kq.z, kq.w};
    float2 sp[ZC_R];
#pragma unroll
    for (int r = 0; r < ZC_R; ++r) sp[r] = __fadd2_rn(e[(r - d) * ZC_EP], e[(r + d) * ZC_EP]);
#pragma unroll
    for (int j = 0; j < ZC_G; ++j) {
      const float2 kk = make_float2(k[j], k[j]);
#pragma unroll
      for (int r = 0; r < ZC_R; ++r) acc[j][r] = __ffma2_rn(kk, sp[r], acc[j][r]);
    }
  }
}

__global__ void __launch_bounds__(ZC_NT, ZC_CTAS) zconv_kernel(ZconvArgs a) {
  extern __shared__ float4 smem4[];
  const int MP = a.dz;
  const int KP = a.dz * ZC_G + 4;  // floats per staged column of a group (16-byte multiple, conflict-free)
  const int erows = a.zc + 2 * MP;
  float2* E = reinterpret_cast<float2*>(smem4);
  float* Kb = reinterpret_cast<float*>(E + (size_t)erows * ZC_EP);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // a warp: 8 columns x 4 plane groups (the 4 lanes of a column share its taps)
  const int c = (warp & 3) * 8 + (lane & 7);
  const int zg = (warp >> 2) * 4 + (lane >> 3);
  // written: the planes z0 .. z0 + nzb - 1; read: the field's planes
  // zi .. zi + nzi - 1 (the spectrum vanishes on the others, which the
  // pruned forward passes leave as they were)
  int z0 = 0, nzb = a.nz, zi = 0, nzi = a.nz;
  if (a.out_box) {
    z0 = a.out_box[4];
    nzb = box_len(a.out_box[4], a.out_box[5]);
  }
  if (a.in_box) {
    zi = a.in_box[4];
    nzi = box_len(a.in_box[4], a.in_box[5]);
  }
  // the box's planes in units of at most zc planes (what shared memory
  // holds), evened out: zce planes per unit, a multiple of 4
  const int64_t ntiles = (a.plane + ZC_C - 1) / ZC_C;
  const int nchunks = (nzb + a.zc - 1) / a.zc;
  const int zce = nchunks > 0 ? (((nzb + nchunks - 1) / nchunks + 3) & ~3) : a.zc;
  const int64_t units = ntiles * nchunks;

  // taps of group g (a compile-time index into the parameter array keeps it
  // out of local memory)
  auto taps_of = [&](int g) {
    int t = 0;
#pragma unroll
    for (int i = 0; i < CK_MAX_SHELLS / ZC_G; ++i)
      if (i == g) t = a.taps[i];
    return t;
  };
  auto stage_k = [&](int64_t i0, int g, int buf) {
    float* kb = Kb + buf * (ZC_C * KP);
    const int nq = taps_of(g) * (ZC_G / 4);  // 16-byte pieces per column: ZC_G floats per tap
    for (int idx = tid; idx < ZC_C * nq; idx += ZC_NT) {
      const int cc = idx / nq, q = idx - (idx / nq) * nq;
      const int64_t i = i0 + cc;
      const bool ok = i < a.plane;
      int64_t off = 0;
      if (ok) {
        const int ky = (int)(i / a.px), kx = (int)(i - (int64_t)ky * a.px);
        const int kyf = min(ky, a.ny - ky);
        off = (int64_t)g * a.group_stride + ((int64_t)kyf * a.px + kx) * (a.dz * ZC_G) + q * 4;
      }
      cp_async16(kb + cc * KP + q * 4, ok ? a.table + off : a.table, ok);
    }
  };

  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t tile = u / nchunks;
    const int ch = (int)(u - tile * nchunks);
    const int64_t i0 = tile * ZC_C;
    const int q0 = ch * zce;  // first output plane of the unit, relative to z0
    const int zcn = min(zce, nzb - q0);
    __syncthreads();  // the previous unit's reads of E and the tap buffers are done
    // E[i] = D at plane z0 + q0 + i - MP (mod n_z), zero outside the field's
    // planes; the passes read rows below ((zcn + 3) & ~3) + 2 MP
    const int rows = min(erows, ((zcn + 3) & ~3) + 2 * MP);
    for (int idx = tid; idx < rows * (ZC_C / 2); idx += ZC_NT) {
      const int i = idx / (ZC_C / 2), cp = idx - (idx / (ZC_C / 2)) * (ZC_C / 2);
      int pl = (z0 + q0 + i - MP) % a.nz;
      if (pl < 0) pl += a.nz;
      int rel = pl - zi;
      if (rel < 0) rel += a.nz;
      const bool ok = rel < nzi && i0 + 2 * cp < a.plane;
      cp_async16(E + i * ZC_EP + 2 * cp, ok ? a.spec + (int64_t)pl * a.plane + i0 + 2 * cp : a.spec, ok);
    }
    stage_k(i0, a.g0, 0);
    cp_async_commit();
    for (int g = a.g0; g < a.g1; ++g) {
      const int buf = (g - a.g0) & 1;
      if (g + 1 < a.g1) {
        stage_k(i0, g + 1, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const float* kc = Kb + buf * (ZC_C * KP) + c * KP;
      const int taps = taps_of(g);
      for (int qb = zg * ZC_R; qb < zcn; qb += ZC_PASS) {
        float2 acc[ZC_G][ZC_R];
#pragma unroll
        for (int j = 0; j < ZC_G; ++j)
#pragma unroll
          for (int r = 0; r < ZC_R; ++r) acc[j][r] = make_float2(0.f, 0.f);
        const float2* e = E + (MP + qb) * ZC_EP + c;  // row of plane qb
        switch (taps) {
          case 4: zconv_taps<4>(e, kc, acc); break;
          case 8: zconv_taps<8>(e, kc, acc); break;
          case 12: zconv_taps<12>(e, kc, acc); break;
          case 16: zconv_taps<16>(e, kc, acc); break;
          case 20: zconv_taps<20>(e, kc, acc); break;
          case 24: zconv_taps<24>(e, kc, acc); break;
          case 28: zconv_taps<28>(e, kc, acc); break;
          default: zconv_taps<32>(e, kc, acc); break;
        }
        const bool col_ok = i0 + c < a.plane;
#pragma unroll
        for (int j = 0; j < ZC_G; ++j) {
          const int s = g * ZC_G + j;
          if (s < a.shell0 || s >= a.shell0 + a.nshells || !col_ok) continue;
          float2* o = a.out + (int64_t)(s - a.shell0) * a.out_stride + (int64_t)(z0 + q0 + qb) * a.plane + i0 + c;
#pragma unroll
          for (int r = 0; r < ZC_R; ++r)
            if (qb + r < zcn) o[(int64_t)r * a.plane] = acc[j][r];
        }
      }
      __syncthreads();  // this group's tap buffer is restaged two groups later
    }
  }
}

// The table from the FP64 (x, y) cosine sums A2[s][d][kyf][kx] (kyf < oy,
// kx < ox) of the kernel-spectrum build.
__global__ void zconv_table_kernel(const double* __restrict__ A2, float* __restrict__ table, int ns, int H1, int oy,
                                   int ox, int px, int dz, int groups, double scale) {
  const int64_t total = (int64_t)groups * oy * px * dz * ZC_G;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % ZC_G);
    const int d = (int)((t / ZC_G) % dz);
    const int64_t col = (t / ((int64_t)ZC_G * dz)) % ((int64_t)oy * px);
    const int g = (int)(t / ((int64_t)ZC_G * dz * oy * px));
    const int kyf = (int)(col / px), kx = (int)(col % px);
    const int s = g * ZC_G + j;
    double v = 0.0;
    if (s < ns && kx < ox && d < H1) v = A2[(((int64_t)s * H1 + d) * oy + kyf) * ox + kx] * scale * (d == 0 ? 0.5 : 1.0);
    table[t] = (float)v;
  }
}

}  // namespace

// Taps per column (dz) and per group of shells (taps[g]) for the shells'
// largest |m_z|; dz = 0 when the direct route does not apply (more than 32
// taps: the transform route is then the cheaper one).
void zconv_layout(Plan& p) {
  p.kz_dz = 0;
  p.kz_groups = (p.ns + ZC_G - 1) / ZC_G;
  int mz_all = 0;
  for (int g = 0; g < p.kz_groups; ++g) {
    int mz = 0;
    for (int s = g * ZC_G; s < std::min(p.ns, (g + 1) * ZC_G); ++s) {
      const std::vector<int>& o = p.offsets[(size_t)s];
      for (size_t i = 2; i < o.size(); i += 3) mz = std::max(mz, std::abs(o[i]));
    }
    p.kz_taps[g] = (mz + 1 + 3) / 4 * 4;
    mz_all = std::max(mz_all, mz);
  }
  const int dz = (mz_all + 1 + 3) / 4 * 4;
  if (dz > 32) return;
  p.kz_dz = dz;
  p.kz_group_stride = (int64_t)p.oct[1] * p.px * dz * ZC_G;
}

size_t zconv_table_bytes(const Plan& p) {
  return p.kz_dz > 0 ? (size_t)p.kz_groups * (size_t)p.kz_group_stride * sizeof(float) : 0;
}

cudaError_t launch_zconv_table(const Plan& p, const double* A2, cudaStream_t st) {
  if (p.kz_dz == 0 || !p.kzt) return cudaSuccess;
  const unsigned blocks = (unsigned)std::max(1, p.sm_count * 8);
  zconv_table_kernel<<<blocks, 256, 0, st>>>(A2, p.kzt, p.ns, p.H + 1, p.oct[1], p.oct[0], p.px, p.kz_dz,
                                             p.kz_groups, 1.0 / ((double)p.grid.n[0] * p.grid.n[1]));
  return cudaGetLastError();
}

void launch_zconv(const Plan& p, const float2* spec, int shell0, int nshells, float2* out, int64_t out_stride,
                  const int* in_box, const int* out_box, cudaStream_t st) {
  const int nz = p.grid.n[2];
  ZconvArgs a{};
  a.spec = spec;
  a.out = out;
  a.out_stride = out_stride;
  a.table = p.kzt;
  a.group_stride = p.kz_group_stride;
  a.plane = (int64_t)p.grid.n[1] * p.px;
  a.in_box = in_box;
  a.out_box = out_box;
  a.px = p.px;
  a.ny = p.grid.n[1];
  a.nz = nz;
  a.dz = p.kz_dz;
  a.shell0 = shell0;
  a.nshells = nshells;
  a.g0 = shell0 / ZC_G;
  a.g1 = (shell0 + nshells + ZC_G - 1) / ZC_G;
  for (int g = 0; g < p.kz_groups; ++g) a.taps[g] = p.kz_taps[g];
  // the most planes per unit (up to the axis) that keep three CTAs per SM;
  // the kernel evens the box's planes out over the units they take
  int zc = (nz + 3) / 4 * 4;
  while (zc > 4 && zconv_smem(a.dz, zc) > ZC_SMEM_CAP) zc -= 4;
  a.zc = zc;
  const size_t smem = zconv_smem(a.dz, zc);
  if (smem > 48 * 1024) cudaFuncSetAttribute(zconv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t ntiles = (a.plane + ZC_C - 1) / ZC_C;
  const int64_t units = ntiles * ((nz + zc - 1) / zc);  // at most (the box may hold fewer planes)
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)ZC_CTAS * p.sm_count));
  zconv_kernel<<<grid, ZC_NT, smem, st>>>(a);
}

}  // namespace ck
