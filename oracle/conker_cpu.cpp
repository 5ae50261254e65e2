// conker_cpu.cpp -- FP64 CPU engine of the same oracle definitions, in C++17
// with OpenMP, for timing the method on the host cores at full size.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/ and bench.py's CPU-baseline and
// reference legs call it.  It shares no code, table or constant with the CUDA
// library; the numpy oracle (conker_oracle.py) stays the pinned authority and
// this engine is checked against it to 1e-12 on small grids.
//
// What it computes, in the paper's order (Sec. 2), with the numpy oracle's
// readings:
//  * mapping (Sec. 2.2): nearest-grid-point histograms D, R, a float32
//    coordinate in cell k iff e_k <= x < e_{k+1}, e_k = fl64(origin +
//    fl64(k g)); periodic grids wrap k mod n, other grids drop and count;
//    alpha = sum D / sum R (or a given alpha), N = D - alpha R, Rt = alpha R;
//  * kernels (Sec. 2.3): the integer offsets m of shell s, centre-bin rule
//    (s - w/2) <= |m| g < (s + w/2) or intersect rule dmin^2 <= s^2 < dmax^2,
//    squares compared in FP64;
//  * convolution (Sec. 2.4, Eqs. 9-10): W_s(r) = sum_m N(r + m),
//    B_s(r) = sum_m Rt(r + m), either directly in real space (engine 0;
//    circular on periodic grids, zero outside otherwise) or by the
//    convolution theorem with an FP64 FFT written here (engine 1; the
//    circular convolution, equal to the linear one when the occupied cells
//    keep clear of the faces by the kernel's reach): the transform of
//    Z = N + i Rt, times the kernel's transform K^_s (real, K_s being even:
//    separable FP64 cosine sums over its offsets), transformed back, gives
//    W_s + i B_s at once, both being real; the inverse transform is carried
//    to the end only inside the box of occupied cells, where they are read;
//  * summation (Sec. 2.5, Eqs. 11-13): for every multiset s_1 <= .. <=
//    s_{n-1} (lexicographic), num = sum_r N prod W_{s_i},
//    den = sum_r Rt prod B_{s_i}, and the sums of |terms|.  Cells where N and
//    Rt both vanish add nothing and are skipped: the banks are kept only at
//    the occupied cells.
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

namespace {

using cplx = std::complex<double>;

struct Grid {
  int n[3];
  double origin[3];
  double cell;
  int periodic;
  int64_t cells() const { return (int64_t)n[0] * n[1] * n[2]; }
};

// The cell of a float32 coordinate on one axis (edge rule above), or
// INT64_MIN for a non-finite coordinate.
int64_t cell_of(float xf, double origin, double g) {
  const double x = (double)xf;
  if (!std::isfinite(x)) return INT64_MIN;
  int64_t k = (int64_t)floor((x - origin) / g);
  for (int it = 0; it < 8; ++it) {
    const double lo = origin + (double)k * g, hi = origin + (double)(k + 1) * g;
    if (x < lo) --k;
    else if (x >= hi) ++k;
    else return k;
  }
  return k;
}

// Histogram of points per cell (z-major layout), returns the dropped count.
int64_t histogram(const Grid& G, const float* x, const float* y, const float* z, int64_t np, std::vector<double>& H) {
  H.assign((size_t)G.cells(), 0.0);
  int64_t dropped = 0;
  for (int64_t i = 0; i < np; ++i) {
    const float c[3] = {x[i], y[i], z[i]};
    int64_t k[3];
    bool in = true;
    for (int a = 0; a < 3; ++a) {
      k[a] = cell_of(c[a], G.origin[a], G.cell);
      if (k[a] == INT64_MIN) { in = false; break; }
      if (G.periodic) {
        k[a] %= G.n[a];
        if (k[a] < 0) k[a] += G.n[a];
      } else if (k[a] < 0 || k[a] >= G.n[a]) {
        in = false;
      }
    }
    if (!in) { ++dropped; continue; }
    H[(size_t)((k[2] * G.n[1] + k[1]) * G.n[0] + k[0])] += 1.0;
  }
  return dropped;
}

std::vector<int> shell_offsets(double s, double w, double g, int rule) {
  std::vector<int> out;
  const double outer = rule == 0 ? s + 0.5 * w : s + g;
  const int h = (int)ceil(outer / g) + 1;
  const double lo = std::max(s - 0.5 * w, 0.0), hi = s + 0.5 * w;
  for (int mx = -h; mx <= h; ++mx)
    for (int my = -h; my <= h; ++my)
      for (int mz = -h; mz <= h; ++mz) {
        bool in;
        if (rule == 0) {
          const double d2 = (double)(mx * mx + my * my + mz * mz) * g * g;
          in = d2 >= lo * lo && d2 < hi * hi;
        } else {
          auto nr = [](int a) { const double t = std::max(fabs((double)a) - 0.5, 0.0); return t * t; };
          auto fr = [](int a) { const double t = fabs((double)a) + 0.5; return t * t; };
          const double dmin2 = (nr(mx) + nr(my) + nr(mz)) * g * g, dmax2 = (fr(mx) + fr(my) + fr(mz)) * g * g;
          in = dmin2 <= s * s && s * s < dmax2;
        }
        if (in) { out.push_back(mx); out.push_back(my); out.push_back(mz); }
      }
  return out;
}

// ---------------------------------------------------------------------------
// FP64 FFT of lines (lengths with the prime factors 2, 3, 5): a Stockham
// self-sorting decimation-in-frequency transform, one radix per stage,
// ping-ponging between two buffers, e^{sign 2 pi i jk / n}.  A stage of
// radix r over sequences of length L = r m, `s` of them interleaved, maps
//   y[q + s (r p + k)] = w_L^{p k} sum_j x[q + s (p + j m)] w_r^{j k},
// so that the m-point transform of sequence q + s k gives the outputs
// k + r d in natural order.  NB lines are transformed together, element i of
// line b at buf[i NB + b], so that every load and store moves NB values.

constexpr int NB = 8;

struct Stage {
  int r, m, s;
  std::vector<cplx> tw;  // tw[p r + k] = w_L^{p k} (forward sign)
};

struct Line {
  int n = 0;
  std::vector<Stage> st;
};

Line make_line(int n) {
  Line L;
  L.n = n;
  std::vector<int> radix;
  int m = n;
  for (int r : {4, 2, 3, 5})
    while (m % r == 0) {
      radix.push_back(r);
      m /= r;
    }
  int len = n, s = 1;
  for (int r : radix) {
    Stage S;
    S.r = r;
    S.m = len / r;
    S.s = s;
    S.tw.resize((size_t)len);
    for (int p = 0; p < S.m; ++p)
      for (int k = 0; k < r; ++k) {
        const double a = -2.0 * M_PI * (double)(((int64_t)p * k) % len) / (double)len;
        S.tw[(size_t)(p * r + k)] = cplx(cos(a), sin(a));
      }
    L.st.push_back(std::move(S));
    len /= r;
    s *= r;
  }
  return L;
}

// NB interleaved lines of length n in x (transformed in place); work: n NB.
void fft_lines(const Line& L, cplx* x, cplx* work, int sign) {
  cplx* a = x;
  cplx* b = work;
  const double sg = sign < 0 ? 1.0 : -1.0;  // conjugate the forward roots for the inverse
  for (const Stage& S : L.st) {
    const int r = S.r, m = S.m, s = S.s;
    cplx wr[25];
    for (int j = 0; j < r; ++j)
      for (int k = 0; k < r; ++k) {
        const double ang = -2.0 * M_PI * (double)((j * k) % r) / (double)r;
        wr[j * r + k] = cplx(cos(ang), sg * sin(ang));
      }
    for (int p = 0; p < m; ++p) {
      cplx t[5];
      for (int k = 0; k < r; ++k) {
        const cplx w = S.tw[(size_t)(p * r + k)];
        t[k] = cplx(w.real(), sg * w.imag());
      }
      for (int q = 0; q < s; ++q) {
        const cplx* src = a + (size_t)(q + s * p) * NB;
        const size_t jstep = (size_t)s * m * NB;
        cplx* dst = b + (size_t)(q + s * r * p) * NB;
        const size_t kstep = (size_t)s * NB;
        if (r == 4) {
          const double ii = sign < 0 ? -1.0 : 1.0;  // w_4 = e^{sign i pi / 2}
          for (int e = 0; e < NB; ++e) {
            const cplx x0 = src[e], x1 = src[jstep + e], x2 = src[2 * jstep + e], x3 = src[3 * jstep + e];
            const cplx s02 = x0 + x2, d02 = x0 - x2, s13 = x1 + x3, d13 = x1 - x3;
            const cplx jd13(-ii * d13.imag(), ii * d13.real());  // d13 times e^{sign i pi / 2}
            dst[e] = (s02 + s13) * t[0];
            dst[kstep + e] = (d02 + jd13) * t[1];
            dst[2 * kstep + e] = (s02 - s13) * t[2];
            dst[3 * kstep + e] = (d02 - jd13) * t[3];
          }
        } else if (r == 2) {
          for (int e = 0; e < NB; ++e) {
            const cplx x0 = src[e], x1 = src[jstep + e];
            dst[e] = (x0 + x1) * t[0];
            dst[kstep + e] = (x0 - x1) * t[1];
          }
        } else {
          for (int e = 0; e < NB; ++e) {
            cplx v[5];
            for (int j = 0; j < r; ++j) v[j] = src[(size_t)j * jstep + e];
            for (int k = 0; k < r; ++k) {
              cplx acc(0.0, 0.0);
              for (int j = 0; j < r; ++j) acc += v[j] * wr[j * r + k];
              dst[(size_t)k * kstep + e] = acc * t[k];
            }
          }
        }
      }
    }
    std::swap(a, b);
  }
  if (a != x) std::copy(a, a + (size_t)L.n * NB, x);
}

// In-place 3D transform of a z-major array (nz, ny, nx): axis by axis, NB
// lines at a time (adjacent rows for x; adjacent x columns for y and z, so
// that each gathered row is NB contiguous values), groups in parallel.
void fft3(const Grid& G, cplx* A, int sign) {
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const Line Lx = make_line(nx), Ly = make_line(ny), Lz = make_line(nz);
  const int nmax = std::max(nx, std::max(ny, nz));
  const int64_t rows = (int64_t)ny * nz;
#pragma omp parallel
  {
    std::vector<cplx> buf((size_t)nmax * NB), work((size_t)nmax * NB);
#pragma omp for schedule(static)
    for (int64_t r0 = 0; r0 < rows; r0 += NB) {
      const int nb = (int)std::min<int64_t>(NB, rows - r0);
      for (int i = 0; i < nx; ++i)
        for (int e = 0; e < NB; ++e) buf[(size_t)i * NB + e] = e < nb ? A[(r0 + e) * nx + i] : cplx(0.0, 0.0);
      fft_lines(Lx, buf.data(), work.data(), sign);
      for (int i = 0; i < nx; ++i)
        for (int e = 0; e < nb; ++e) A[(r0 + e) * nx + i] = buf[(size_t)i * NB + e];
    }
    // y and z: groups of NB adjacent x columns
    const int gx = (nx + NB - 1) / NB;
    auto columns = [&](const Line& L, int len, int64_t stride, cplx* base, int nb) {
      for (int j = 0; j < len; ++j)
        for (int e = 0; e < NB; ++e) buf[(size_t)j * NB + e] = e < nb ? base[j * stride + e] : cplx(0.0, 0.0);
      fft_lines(L, buf.data(), work.data(), sign);
      for (int j = 0; j < len; ++j)
        for (int e = 0; e < nb; ++e) base[j * stride + e] = buf[(size_t)j * NB + e];
    };
#pragma omp for schedule(static)
    for (int64_t t = 0; t < (int64_t)nz * gx; ++t) {
      const int64_t zz = t / gx;
      const int x0 = (int)(t % gx) * NB;
      columns(Ly, ny, nx, A + zz * (int64_t)ny * nx + x0, std::min(NB, nx - x0));
    }
#pragma omp for schedule(static)
    for (int64_t t = 0; t < (int64_t)ny * gx; ++t) {
      const int64_t yy = t / gx;
      const int x0 = (int)(t % gx) * NB;
      columns(Lz, nz, (int64_t)ny * nx, A + yy * nx + x0, std::min(NB, nx - x0));
    }
  }
}

// Inverse transform of a z-major array needed only inside the box
// [x0..x1] x [y0..y1] x [z0..z1]: z lines over every column, then y lines of
// the planes z0..z1, then x lines of the rows inside the box; elsewhere the
// array is left partly transformed.
void ifft3_box(const Grid& G, cplx* A, const int* box) {
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const Line Lx = make_line(nx), Ly = make_line(ny), Lz = make_line(nz);
  const int nmax = std::max(nx, std::max(ny, nz));
  const int y0 = box[2], y1 = box[3], z0 = box[4], z1 = box[5];
  const int nyb = y1 - y0 + 1, nzb = z1 - z0 + 1;
  if (nyb <= 0 || nzb <= 0) return;
  const int gx = (nx + NB - 1) / NB;
#pragma omp parallel
  {
    std::vector<cplx> buf((size_t)nmax * NB), work((size_t)nmax * NB);
    auto columns = [&](const Line& L, int len, int64_t stride, cplx* base, int nb) {
      for (int j = 0; j < len; ++j)
        for (int e = 0; e < NB; ++e) buf[(size_t)j * NB + e] = e < nb ? base[j * stride + e] : cplx(0.0, 0.0);
      fft_lines(L, buf.data(), work.data(), +1);
      for (int j = 0; j < len; ++j)
        for (int e = 0; e < nb; ++e) base[j * stride + e] = buf[(size_t)j * NB + e];
    };
#pragma omp for schedule(static)
    for (int64_t t = 0; t < (int64_t)ny * gx; ++t) {
      const int64_t yy = t / gx;
      const int x0 = (int)(t % gx) * NB;
      columns(Lz, nz, (int64_t)ny * nx, A + yy * nx + x0, std::min(NB, nx - x0));
    }
#pragma omp for schedule(static)
    for (int64_t t = 0; t < (int64_t)nzb * gx; ++t) {
      const int64_t zz = z0 + t / gx;
      const int x0 = (int)(t % gx) * NB;
      columns(Ly, ny, nx, A + zz * (int64_t)ny * nx + x0, std::min(NB, nx - x0));
    }
    const int64_t rows = (int64_t)nyb * nzb;
#pragma omp for schedule(static)
    for (int64_t r0 = 0; r0 < rows; r0 += NB) {
      const int nb = (int)std::min<int64_t>(NB, rows - r0);
      int64_t roff[NB];
      for (int e = 0; e < NB; ++e) {
        const int64_t c = r0 + std::min(e, nb - 1);
        roff[e] = ((z0 + c / nyb) * (int64_t)ny + y0 + c % nyb) * nx;
      }
      for (int i = 0; i < nx; ++i)
        for (int e = 0; e < NB; ++e) buf[(size_t)i * NB + e] = e < nb ? A[roff[e] + i] : cplx(0.0, 0.0);
      fft_lines(Lx, buf.data(), work.data(), +1);
      for (int i = 0; i < nx; ++i)
        for (int e = 0; e < nb; ++e) A[roff[e] + i] = buf[(size_t)i * NB + e];
    }
  }
}

// The transform of a shell kernel K (0/1 on its offsets, even in every
// axis), real: sum over the offsets m >= 0 per axis of the product of
// cos(2 pi k_a m_a / n_a), each weighted 1 for m_a = 0 and 2 otherwise,
// in three separable passes (x, then y, then z), FP64.  Out: (nz, ny, nx).
void kernel_spectrum(const Grid& G, const std::vector<int>& o, std::vector<double>& out) {
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  int h = 0;
  for (int v : o) h = std::max(h, std::abs(v));
  const int H1 = h + 1;
  std::vector<double> Kc((size_t)H1 * H1 * H1, 0.0);  // [mz][my][mx], m >= 0
  for (size_t t = 0; t < o.size(); t += 3)
    if (o[t] >= 0 && o[t + 1] >= 0 && o[t + 2] >= 0)
      Kc[((size_t)o[t + 2] * H1 + o[t + 1]) * H1 + o[t]] = 1.0;
  auto table = [&](int n, std::vector<double>& c) {
    c.assign((size_t)n * H1, 0.0);
    for (int k = 0; k < n; ++k)
      for (int m = 0; m < H1; ++m)
        c[(size_t)k * H1 + m] = (m == 0 ? 1.0 : 2.0) * cos(2.0 * M_PI * (double)(((int64_t)k * m) % n) / (double)n);
  };
  std::vector<double> cx, cy, cz;
  table(nx, cx);
  table(ny, cy);
  table(nz, cz);
  std::vector<double> A1((size_t)H1 * H1 * nx), A2((size_t)H1 * ny * nx);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < (int64_t)H1 * H1 * nx; ++t) {
    const int kx = (int)(t % nx);
    const int64_t zy = t / nx;
    double acc = 0.0;
    for (int m = 0; m < H1; ++m) acc += Kc[(size_t)zy * H1 + m] * cx[(size_t)kx * H1 + m];
    A1[(size_t)t] = acc;
  }
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < (int64_t)H1 * ny * nx; ++t) {
    const int kx = (int)(t % nx), ky = (int)((t / nx) % ny);
    const int64_t mz = t / ((int64_t)ny * nx);
    double acc = 0.0;
    for (int m = 0; m < H1; ++m) acc += A1[((size_t)mz * H1 + m) * nx + kx] * cy[(size_t)ky * H1 + m];
    A2[(size_t)t] = acc;
  }
  out.resize((size_t)G.cells());
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < G.cells(); ++t) {
    const int64_t kyx = t % ((int64_t)ny * nx);
    const int kz = (int)(t / ((int64_t)ny * nx));
    double acc = 0.0;
    for (int m = 0; m < H1; ++m) acc += A2[(size_t)m * ny * nx + kyx] * cz[(size_t)kz * H1 + m];
    out[(size_t)t] = acc;
  }
}

// ---------------------------------------------------------------------------
// multisets s_1 <= .. <= s_k over ns shells, lexicographic
void multisets(int ns, int k, std::vector<std::vector<int>>& out) {
  out.clear();
  std::vector<int> s((size_t)k, 0);
  if (k == 0) { out.push_back(s); return; }
  while (true) {
    out.push_back(s);
    int i = k - 1;
    while (i >= 0 && s[(size_t)i] == ns - 1) --i;
    if (i < 0) break;
    const int v = s[(size_t)i] + 1;
    for (int j = i; j < k; ++j) s[(size_t)j] = v;
  }
}

}  // namespace

extern "C" {

// Number of OpenMP threads the engine will use.
int cko_threads(void) { return omp_get_max_threads(); }

// The whole path for one catalog.  grid: n[3], origin[3], cell, periodic;
// shells: n_shells radii, width, rule (0 centre-bin, 1 intersect); data and
// randoms float32 positions; order_mask bit n -> order n (2..5); engine 0
// direct, 1 FFT; alpha <= 0: sum D / sum R, else the given value; owned_z0 <
// owned_z1: the sums over planes owned_z0 <= z < owned_z1 only.  Outputs, per
// order in multiset order, packed order after order (n = 2 first): num, den,
// anum, aden (sums of |terms|); alpha_out, dropped[2].  Returns 0, or 1 for
// bad arguments (empty randoms, unsupported length).
int cko_correlate(const int* n, const double* origin, double cell, int periodic, int n_shells, const double* radius,
                  double width, int rule, const float* dx, const float* dy, const float* dz, int64_t nd,
                  const float* rx, const float* ry, const float* rz, int64_t nr, int order_mask, int engine,
                  double alpha_in, int owned_z0, int owned_z1, double* num, double* den, double* anum, double* aden,
                  double* alpha_out, int64_t* dropped) {
  Grid G;
  for (int a = 0; a < 3; ++a) {
    G.n[a] = n[a];
    G.origin[a] = origin[a];
    int m = n[a];
    for (int p : {2, 3, 5})
      while (m % p == 0) m /= p;
    if (n[a] < 1 || (engine == 1 && m != 1)) return 1;
  }
  G.cell = cell;
  G.periodic = periodic;
  const int64_t nc = G.cells();
  const int ns = n_shells;
  std::vector<double> D, R;
  dropped[0] = histogram(G, dx, dy, dz, nd, D);
  dropped[1] = histogram(G, rx, ry, rz, nr, R);
  double sd = 0.0, sr = 0.0;
  for (int64_t i = 0; i < nc; ++i) { sd += D[(size_t)i]; sr += R[(size_t)i]; }
  if (!(alpha_in > 0.0) && !(sr > 0.0)) return 1;
  const double alpha = alpha_in > 0.0 ? alpha_in : sd / sr;
  *alpha_out = alpha;
  std::vector<double> N((size_t)nc), Rt((size_t)nc);
  for (int64_t i = 0; i < nc; ++i) {
    N[(size_t)i] = D[(size_t)i] - alpha * R[(size_t)i];
    Rt[(size_t)i] = alpha * R[(size_t)i];
  }
  // the occupied cells (W_0 or B_0 nonzero) inside the owned planes
  const int64_t plane = (int64_t)G.n[0] * G.n[1];
  const int z0 = owned_z0 < owned_z1 ? owned_z0 : 0, z1 = owned_z0 < owned_z1 ? owned_z1 : G.n[2];
  std::vector<int64_t> occ;
  for (int64_t i = (int64_t)z0 * plane; i < (int64_t)z1 * plane; ++i)
    if (N[(size_t)i] != 0.0 || Rt[(size_t)i] != 0.0) occ.push_back(i);
  const int64_t no = (int64_t)occ.size();
  // banks at the occupied cells: W[s][j], B[s][j]
  std::vector<double> W((size_t)ns * no), B((size_t)ns * no);
  std::vector<std::vector<int>> offs;
  for (int s = 0; s < ns; ++s) offs.push_back(shell_offsets(radius[s], width, cell, rule));
  if (engine == 0) {
    for (int s = 0; s < ns; ++s) {
      const std::vector<int>& o = offs[(size_t)s];
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < no; ++j) {
        const int64_t i = occ[(size_t)j];
        const int ix = (int)(i % G.n[0]), iy = (int)((i / G.n[0]) % G.n[1]), iz = (int)(i / plane);
        double w = 0.0, b = 0.0;
        for (size_t t = 0; t < o.size(); t += 3) {
          int jx = ix + o[t], jy = iy + o[t + 1], jz = iz + o[t + 2];
          if (periodic) {
            jx = ((jx % G.n[0]) + G.n[0]) % G.n[0];
            jy = ((jy % G.n[1]) + G.n[1]) % G.n[1];
            jz = ((jz % G.n[2]) + G.n[2]) % G.n[2];
          } else if (jx < 0 || jx >= G.n[0] || jy < 0 || jy >= G.n[1] || jz < 0 || jz >= G.n[2]) {
            continue;
          }
          const size_t k = (size_t)((int64_t)jz * plane + (int64_t)jy * G.n[0] + jx);
          w += N[k];
          b += Rt[k];
        }
        W[(size_t)s * no + j] = w;
        B[(size_t)s * no + j] = b;
      }
    }
  } else {
    std::vector<cplx> Zh((size_t)nc), K((size_t)nc);
    std::vector<double> Kh;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nc; ++i) Zh[(size_t)i] = cplx(N[(size_t)i], Rt[(size_t)i]);
    fft3(G, Zh.data(), -1);
    const double inv = 1.0 / (double)nc;
    // the occupied cells' box: W and B are needed there only
    int box[6] = {G.n[0], -1, G.n[1], -1, G.n[2], -1};
    for (int64_t j = 0; j < no; ++j) {
      const int64_t i = occ[(size_t)j];
      const int c[3] = {(int)(i % G.n[0]), (int)((i / G.n[0]) % G.n[1]), (int)(i / plane)};
      for (int a = 0; a < 3; ++a) {
        box[2 * a] = std::min(box[2 * a], c[a]);
        box[2 * a + 1] = std::max(box[2 * a + 1], c[a]);
      }
    }
    for (int s = 0; s < ns; ++s) {
      // W + i B = IFFT( FFT(N + i Rt) K^ ) / N_c (K even: its transform K^ is real)
      kernel_spectrum(G, offs[(size_t)s], Kh);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < nc; ++i) K[(size_t)i] = Zh[(size_t)i] * Kh[(size_t)i];
      ifft3_box(G, K.data(), box);
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < no; ++j) {
        const cplx v = K[(size_t)occ[(size_t)j]] * inv;
        W[(size_t)s * no + j] = v.real();
        B[(size_t)s * no + j] = v.imag();
      }
    }
  }
  // product sums of every requested order, per thread then added in thread order
  std::vector<std::vector<std::vector<int>>> sets(6);
  std::vector<int64_t> base(7, 0);
  for (int k = 2; k <= 5; ++k) {
    if ((order_mask >> k) & 1) multisets(ns, k - 1, sets[(size_t)k]);
    base[(size_t)k + 1] = base[(size_t)k] + (int64_t)sets[(size_t)k].size();
  }
  const int64_t total = base[6];
  const int nth = omp_get_max_threads();
  std::vector<double> acc((size_t)nth * 4 * total, 0.0);
#pragma omp parallel
  {
    const int t = omp_get_thread_num();
    double* a = acc.data() + (size_t)t * 4 * total;
    std::vector<double> w((size_t)ns), b((size_t)ns);
#pragma omp for schedule(static)
    for (int64_t j = 0; j < no; ++j) {
      const double n0 = N[(size_t)occ[(size_t)j]], b0 = Rt[(size_t)occ[(size_t)j]];
      for (int s = 0; s < ns; ++s) {
        w[(size_t)s] = W[(size_t)s * no + j];
        b[(size_t)s] = B[(size_t)s * no + j];
      }
      for (int k = 2; k <= 5; ++k) {
        const std::vector<std::vector<int>>& S = sets[(size_t)k];
        for (size_t m = 0; m < S.size(); ++m) {
          double pn = n0, pd = b0;
          for (int s : S[m]) {
            pn *= w[(size_t)s];
            pd *= b[(size_t)s];
          }
          const size_t o = (size_t)(base[(size_t)k] + (int64_t)m);
          a[o] += pn;
          a[total + o] += pd;
          a[2 * total + o] += fabs(pn);
          a[3 * total + o] += fabs(pd);
        }
      }
    }
  }
  for (int64_t o = 0; o < total; ++o) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = 0; t < nth; ++t)
      for (int q = 0; q < 4; ++q) v[q] += acc[(size_t)t * 4 * total + (size_t)q * total + (size_t)o];
    num[o] = v[0];
    den[o] = v[1];
    anum[o] = v[2];
    aden[o] = v[3];
  }
  return 0;
}

}  // extern "C"
