// ck_plan.cu -- host side of a plan: argument validation, the shell offset
// lists (Sec. 2.3), FFT length factorisation and the workspace layout.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "ck_internal.h"

namespace ck {

ck_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CK_OK;
  if (e == cudaErrorMemoryAllocation) return CK_ERR_OOM;
  return CK_ERR_CUDA;
}

int64_t binom(int64_t n, int64_t k) {
  if (k < 0 || k > n) return 0;
  int64_t r = 1;
  for (int64_t i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

bool factor_len(int n, FftLen* out) {
  const RPlan r = rplan(n);
  if (r.nst <= 0) return false;
  FftLen f;
  f.n = n;
  f.nst = r.nst;
  for (int i = 0; i < r.nst; ++i) f.radix[i] = r.r[i];
  *out = f;
  return true;
}

// Integer offsets of one shell under the chosen rule (Sec. 2.3), as a
// flattened (mx, my, mz) list.  center_bin: (s - w/2) <= |m| g < (s + w/2);
// intersect: the sphere of radius s meets the closed cell cube,
// dmin^2 <= s^2 < dmax^2.  All comparisons of squares in FP64.
static std::vector<int> shell_list(double s, double w, double g, int rule) {
  std::vector<int> out;
  const double g2 = g * g;
  const double outer = rule == CK_SHELL_CENTER_BIN ? s + 0.5 * w : s + g;
  const int h = (int)ceil(outer / g) + 1;
  const double lo = std::max(s - 0.5 * w, 0.0);
  const double hi = s + 0.5 * w;
  for (int mx = -h; mx <= h; ++mx)
    for (int my = -h; my <= h; ++my)
      for (int mz = -h; mz <= h; ++mz) {
        bool in;
        if (rule == CK_SHELL_CENTER_BIN) {
          const double d2 = (double)(mx * mx + my * my + mz * mz) * g2;
          in = d2 >= lo * lo && d2 < hi * hi;
        } else {
          auto nr = [](int a) { double t = std::max(fabs((double)a) - 0.5, 0.0); return t * t; };
          auto fr = [](int a) { double t = fabs((double)a) + 0.5; return t * t; };
          const double dmin2 = (nr(mx) + nr(my) + nr(mz)) * g2;
          const double dmax2 = (fr(mx) + fr(my) + fr(mz)) * g2;
          in = dmin2 <= s * s && s * s < dmax2;
        }
        if (in) { out.push_back(mx); out.push_back(my); out.push_back(mz); }
      }
  return out;
}

// Largest dynamic shared memory a CTA may opt in to (227 KB).
constexpr size_t kMaxSmemOptin = 227 * 1024;

static bool finite(double v) { return isfinite(v) != 0; }

ck_status validate_and_layout(const ck_grid* grid, const ck_shells* shells, int max_order,
                              int precision, Plan* p) {
  if (!grid || !shells || !p) return CK_ERR_BAD_POINTER;
  const bool padded = grid->periodic == CK_GRID_PADDED;  // any other nonzero value: periodic
  for (int a = 0; a < 3; ++a) {
    const int n = grid->n[a];
    if (padded) {
      if (n < 2 || n > 512) return CK_ERR_UNSUPPORTED;
    } else {
      if (n < 2 || n > 512 || (n % 2) != 0) return CK_ERR_UNSUPPORTED;
      FftLen f;
      if (!factor_len(n, &f) || !factor_len(n / 2, &f)) return CK_ERR_UNSUPPORTED;
    }
    if (!finite(grid->origin[a])) return CK_ERR_ARG;
  }
  if (!(grid->cell > 0.0) || !finite(grid->cell)) return CK_ERR_ARG;
  if (shells->n_shells < 1 || shells->n_shells > CK_MAX_SHELLS) return CK_ERR_ARG;
  if (!shells->radius) return CK_ERR_BAD_POINTER;
  if (shells->rule != CK_SHELL_CENTER_BIN && shells->rule != CK_SHELL_INTERSECT) return CK_ERR_ARG;
  if (!finite(shells->width) || shells->width < 0.0) return CK_ERR_ARG;
  if (shells->rule == CK_SHELL_CENTER_BIN && !(shells->width > 0.0)) return CK_ERR_ARG;
  for (int s = 0; s < shells->n_shells; ++s)
    if (!(shells->radius[s] > 0.0) || !finite(shells->radius[s])) return CK_ERR_ARG;
  if (max_order < 2 || max_order > CK_MAX_ORDER) return CK_ERR_ARG;
  if (precision != CK_PREC_FP32 && precision != CK_PREC_FP64_SUM && precision != CK_PREC_SPLIT_TF32 &&
      precision != CK_PREC_SPLIT_BF16 && precision != CK_PREC_SPLIT_FP16)
    return CK_ERR_ARG;
  // The packed dense outputs must stay modest.
  int64_t dense = 1;
  for (int k = 1; k < max_order; ++k) dense *= shells->n_shells;
  if (dense > (int64_t)1 << 24) return CK_ERR_ARG;

  p->grid = *grid;
  p->ns = shells->n_shells;
  p->width = shells->width;
  p->rule = shells->rule;
  p->max_order = max_order;
  p->precision = precision;
  p->radius.assign(shells->radius, shells->radius + shells->n_shells);
  p->offsets.clear();
  p->maxoff[0] = p->maxoff[1] = p->maxoff[2] = 0;
  for (int s = 0; s < p->ns; ++s) {
    std::vector<int> o = shell_list(p->radius[s], p->width, grid->cell, p->rule);
    if (o.empty()) return CK_ERR_EMPTY_SHELL;
    for (size_t i = 0; i < o.size(); i += 3)
      for (int a = 0; a < 3; ++a) p->maxoff[a] = std::max(p->maxoff[a], abs(o[i + a]));
    p->offsets.push_back(std::move(o));
  }
  for (int a = 0; a < 3; ++a) p->box_n[a] = grid->n[a];
  if (padded) {
    // the transformed grid: per axis the smallest supported length >= n + reach,
    // so that no offset of a cell in the box wraps onto another cell of the box
    p->grid.periodic = 0;
    for (int a = 0; a < 3; ++a) {
      int m = grid->n[a] + p->maxoff[a];
      FftLen f;
      while (m <= 512 && (m % 2 != 0 || !factor_len(m, &f) || !factor_len(m / 2, &f))) ++m;
      if (m > 512) return CK_ERR_UNSUPPORTED;
      p->grid.n[a] = m;
    }
  }
  // Offsets must stay distinct after wrapping into the FFT box.
  for (int a = 0; a < 3; ++a)
    if (2 * p->maxoff[a] >= p->grid.n[a]) return CK_ERR_KERNEL_TOO_LARGE;
  p->H = std::max(p->maxoff[0], std::max(p->maxoff[1], p->maxoff[2]));

  const int nx = p->grid.n[0], ny = p->grid.n[1], nz = p->grid.n[2];
  p->nc = (int64_t)nx * ny * nz;
  p->field_stride = (p->nc + 63) / 64 * 64;
  p->px = ((nx / 2 + 1) + 3) / 4 * 4;
  p->spec_elems = (int64_t)nz * ny * p->px;
  p->oct[0] = nx / 2 + 1;
  p->oct[1] = ny / 2 + 1;
  p->oct[2] = nz / 2 + 1;
  p->oct_elems = (int64_t)p->oct[0] * p->oct[1] * p->oct[2];
  p->khat_stride = (int64_t)p->px * p->oct[1] * p->oct[2];
  // Mixed precision: one fused pass for the inverse x transform and the
  // tensor-core sums (orders <= 3, <= 16 shells), with no bank kept; beyond
  // that the bank is kept and the blocked product runs on the tensor cores.
  p->fused = false;
  if (precision == CK_PREC_SPLIT_TF32 && max_order <= 3) {
    const int pad = xc_pad_shells(p->ns);
    p->fused = pad > 0 && xc_smem_bytes(nx / 2, pad) <= kMaxSmemOptin;
  }
  p->bank_fields = p->fused ? 1 : p->ns;
  factor_len(nx / 2, &p->fx_half);
  factor_len(ny, &p->fy);
  factor_len(nz, &p->fz);
  int64_t base = 0, dbase = 0;
  for (int n = 0; n <= CK_MAX_ORDER; ++n) {
    p->n_multisets[n] = 0;
    p->multiset_base[n] = 0;
    p->dense_elems[n] = 0;
    p->dense_base[n] = 0;
  }
  for (int n = 2; n <= max_order; ++n) {
    p->n_multisets[n] = binom(p->ns + n - 2, n - 1);
    p->multiset_base[n] = base;
    base += p->n_multisets[n];
    int64_t d = 1;
    for (int k = 1; k < n; ++k) d *= p->ns;
    p->dense_elems[n] = d;
    p->dense_base[n] = dbase;
    dbase += d;
  }
  p->n_multiset_total = base;
  p->dense_total = dbase;
  p->staging_pts = (int64_t)1 << 21;
  // Partial sums of the contraction kernels (doubles); split-TF32 plans that
  // keep the bank need one 128 x TN tile of FP64 per tile and split of at
  // most 16384 cells, the splits filling up to 3 CTAs per SM on any device
  // of up to 256 SMs with as few as one tensor-core tile.
  p->partials_cap = (size_t)1 << 22;
  const bool tensor = precision == CK_PREC_SPLIT_TF32 || precision == CK_PREC_SPLIT_BF16 ||
                      precision == CK_PREC_SPLIT_FP16;
  if (tensor && !p->fused) {
    const int64_t ns = p->ns;
    const int64_t urows = 1 + (max_order >= 3 ? ns : 0) + (max_order >= 4 ? ns * (ns + 1) / 2 : 0);
    const int64_t ucols = ns + (max_order >= 5 ? ns * (ns + 1) / 2 : 0);
    // a stacked tile (at most 128 columns) is twice its list length wide
    const int64_t scols = 2 * ((std::min<int64_t>(ucols, 128) + 15) / 16 * 16);
    const int tn = umma_tile_cols((int)std::min<int64_t>(256, std::max(ucols, scols)));
    const int64_t ntiles = ((urows + umma_tile_rows() - 1) / umma_tile_rows()) * ((ucols + tn - 1) / tn);
    const int64_t splits = std::min<int64_t>((p->nc + 31) / 32, std::max<int64_t>((p->nc + 16383) / 16384, 768));
    p->partials_cap = std::max<size_t>(p->partials_cap, (size_t)(splits * ntiles * umma_tile_rows() * tn));
  }
  // Contraction operand tables: one slot per order mask.
  const int64_t rows = 1 + p->ns + (int64_t)p->ns * (p->ns + 1) / 2;
  const int64_t tiles = ((rows + 63) / 64) * ((rows + 63) / 64);
  // tcgen05 tiles: per 128-row tile, records (int4) and a column list (ints)
  const int64_t rtiles = (rows + 127) / 128;
  const int64_t tc = rtiles * (2 * ((rows + 255) / 256 + 1) + (rows + 1) / 2) + 16;
  p->table_arena_cap = (size_t)(1 << (CK_MAX_ORDER + 1)) * (size_t)(2 * rows + std::max(tiles, tc) + 8) * sizeof(int2);
  zconv_layout(*p);
  return CK_OK;
}

static size_t al(size_t b) { return (b + 255) / 256 * 256; }

// Scratch doubles the separable kernel-spectrum build needs (two passes).
size_t khat_scratch_doubles(const Plan& p) {
  const size_t H1 = (size_t)p.H + 1;
  return (size_t)p.ns * (H1 * H1 * H1 + H1 * H1 * p.oct[0] + H1 * p.oct[1] * p.oct[0]) +
         H1 * (p.oct[0] + p.oct[1] + p.oct[2]);
}

size_t workspace_bytes(const Plan& p) {
  size_t b = 0;
  b += 2 * al((size_t)p.nc * 4);                              // counts D, R
  b += al((size_t)p.field_stride * 4);                         // field
  b += al((size_t)p.spec_elems * 8);                           // spec
  b += al((size_t)p.ns * p.spec_elems * 8);                    // tmp: one scratch spectrum per shell
  b += al((size_t)p.ns * p.khat_stride * 4);                   // khat (padded octants)
  b += al(std::max((size_t)p.bank_fields * p.field_stride * 4, khat_scratch_doubles(p) * 8));  // bank
  b += al(p.partials_cap * 8);                                 // partials
  b += al((size_t)2 * 4 * p.staging_pts * 4);                  // staging: x, y, z, w per slot
  b += al((size_t)p.nc * 8);                                   // fixed-point weight sums
  for (int a = 0; a < 3; ++a) b += al((size_t)(p.grid.n[a] + 1) * 4);  // thresholds
  for (int a = 0; a < 3; ++a) b += 2 * al((size_t)p.grid.n[a] * 8);    // twiddles: full and per-iteration
  b += al((size_t)512 * 8);                                            // twiddle matrix of the K^ z pass
  b += al(sizeof(DevState));
  b += al(sizeof(CatalogRef));
  b += 2 * al((size_t)std::max<int64_t>(p.n_multiset_total, 1) * 8);   // den_raw, sums
  b += al((size_t)3 * std::max<int64_t>(p.dense_total, 1) * 8);        // dense staging
  b += al((size_t)std::max<int64_t>(p.dense_total, 1) * 4);            // dense map
  b += al(p.table_arena_cap);
  b += al(14 * 4);                                                      // support boxes, preparation planes
  b += al((size_t)(CK_MAX_SHELLS + 1) * 4);                             // split-FP16 row maxima
  b += al(zconv_table_bytes(p));                                        // the direct z step's table
  return b;
}

}  // namespace ck
