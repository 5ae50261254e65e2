/*
 * conker.h -- C ABI of a GB300 (sm_103a) implementation of the ConKer
 * n-point correlation hot path (arXiv 2108.00015): mapping (Sec. 2.2),
 * spherical-shell kernels (Sec. 2.3), FFT convolution (Sec. 2.4, Eqs. 9-10)
 * and n-point summation (Sec. 2.5, Eqs. 11-14) for n = 2..5.  Around it:
 * weighted catalogs, zero-padded survey boxes, the equidistant functions
 * (Sec. 2.6), sky coordinates and factorised randoms (Sec. 2.2, Eqs. 3-7),
 * continuous fields and cross-correlation (Secs. 2.7-2.8), per-cell maps
 * (Sec. 4.2) and a batched form.
 *
 * Conventions for every entry point
 *   - Every function returns a ck_status; no exception or abort crosses the
 *     boundary.  CK_OK is 0.
 *   - "device" pointers are CUDA device memory (e.g. a torch CUDA tensor's
 *     data_ptr()); "host or device" pointers are detected with
 *     cudaPointerGetAttributes, and host memory may be pageable or pinned.
 *     Pinned host positions that the device can address are read in place
 *     by the gridding kernel, after the call returns: keep them unchanged
 *     until the stream's work is done, as for any asynchronous copy.
 *   - The caller owns every input and output buffer.  The plan owns its
 *     workspace unless the caller passes one to ck_plan_create.
 *   - Work is ordered on the caller's CUDA stream (NULL = legacy default
 *     stream).  A call returns without synchronising unless an output is in
 *     host memory or an input is in host memory.
 *   - Grids are stored z-major: cell (ix, iy, iz) is element
 *     (iz * n[1] + iy) * n[0] + ix.  Half spectra are complex64 (float2,
 *     re/im) [n[2]][n[1]][spec_pitch] with kx = 0 .. n[0]/2 valid.
 *   - Errors found on the device (a wait that timed out, a zero
 *     denominator, a guard-band violation) are recorded in the plan's device
 *     status word; ck_plan_status() synchronises and returns it.  Calls that
 *     synchronise anyway (host outputs) return it directly.
 */
#ifndef CONKER_H
#define CONKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CK_ABI_VERSION 1
#define CK_MAX_SHELLS 64
#define CK_MAX_ORDER 5

typedef enum ck_status {
  CK_OK = 0,
  CK_ERR_ARG = 1,              /* a size, count or option is out of range       */
  CK_ERR_BAD_POINTER = 2,      /* NULL where required, or wrong memory space    */
  CK_ERR_OOM = 3,              /* device allocation failed / workspace too small */
  CK_ERR_EMPTY_SHELL = 4,      /* a shell contains no lattice offset            */
  CK_ERR_KERNEL_TOO_LARGE = 5, /* periodic axis: 2 max|m| >= n (offsets alias)  */
  CK_ERR_GUARD_BAND = 6,       /* non-periodic: occupied extent + max|m| >= n   */
  CK_ERR_ZERO_DENOM = 7,       /* some den <= 0: those xi entries are NaN       */
  CK_ERR_TIMEOUT = 8,          /* a bounded device wait gave up                 */
  CK_ERR_CUDA = 9,             /* a CUDA runtime call failed                    */
  CK_ERR_UNSUPPORTED = 10,     /* grid axis not a product of 2, 3, 5 or > 512;
                                  precision mode not built                      */
  CK_ERR_NO_RANDOMS = 11,      /* ck_compute before ck_set_randoms              */
  CK_ERR_EMPTY_CATALOG = 12    /* no data (or random) point fell in the grid    */
} ck_status;

/* Shell membership rules (Sec. 2.3).  CENTER_BIN keeps the integer offset m
 * iff (s - w/2) <= |m| g < (s + w/2) (distances between cell centres);
 * INTERSECT keeps m iff the sphere of radius s meets the cell cube:
 * dmin(m)^2 <= s^2 < dmax(m)^2 (width ignored). */
#define CK_SHELL_CENTER_BIN 0
#define CK_SHELL_INTERSECT 1

/* Arithmetic of the product-sum contraction (Sec. 2.5).  FFTs are FP32 in
 * every mode and the cross-block reduction is FP64 in every mode.
 *
 * CK_PREC_FP32 ("plain"): every W_s is written to the plan's bank and the
 * products are FP32 FMAs on the CUDA cores with FP32 partial sums.
 * CK_PREC_SPLIT_TF32 ("mixed"): the products run on the tensor cores with
 * each operand split x = hi + lo into two TF32 numbers (hi*hi + hi*lo +
 * lo*hi, FP32 accumulation over up to 512 cells, FP32 over 16-32 such
 * sums, FP64 beyond).  For max_order <= 3 and at most 16 shells they are
 * fused with the last inverse FFT pass and no bank is kept; otherwise the
 * bank is kept and the blocked product of every order runs on the tensor
 * cores. */
typedef enum ck_precision {
  CK_PREC_FP32 = 0,       /* plain: FP32 CUDA-core products and partial sums */
  CK_PREC_SPLIT_BF16 = 1, /* reserved: tensor-core split-BF16 operands       */
  CK_PREC_SPLIT_FP16 = 2, /* reserved: tensor-core split-FP16 operands       */
  CK_PREC_FP64_SUM = 3,   /* FP64 products and sums (reference contraction)  */
  CK_PREC_SPLIT_TF32 = 4  /* mixed: tensor-core split-TF32 sums              */
} ck_precision;

/* A grid of n[0] x n[1] x n[2] cubic cells of side `cell`, lower corner
 * `origin` (Sec. 2.2: grid spacing g_s).  periodic:
 *  CK_GRID_PERIODIC (1, or any value other than 0 and 2): a periodic box
 *     (circular convolution);
 *  0: a survey box, cells outside it count as 0 (linear convolution); the
 *     transforms run on the box itself, so the occupied cells plus the
 *     kernel's reach must fit in it (CK_ERR_GUARD_BAND otherwise);
 *  CK_GRID_PADDED (2): a survey box as for 0, transformed on a zero-padded
 *     grid of, per axis, the smallest supported length >= n[a] + max|m_a|
 *     (the kernel's reach), so no guard band applies; n[a] is then any
 *     size >= 2 whose padded length exists (<= 512).
 * Otherwise each n[a] must be even, <= 512 and have no prime factor other
 * than 2, 3, 5.  Points outside the box are dropped and counted (0 and 2). */
#define CK_GRID_PERIODIC 1
#define CK_GRID_PADDED 2
typedef struct ck_grid {
  int32_t n[3];
  double origin[3];
  double cell;
  int32_t periodic;
} ck_grid;

/* The radial bins (Sec. 2.3 / Sec. 3): n_shells radii (host array, copied at
 * plan creation), a common width, and a membership rule. */
typedef struct ck_shells {
  int32_t n_shells;
  const double* radius;
  double width;
  int32_t rule;
} ck_shells;

typedef struct ck_plan ck_plan;

typedef struct ck_plan_info {
  int64_t n_cells;                 /* cells of the transformed grid (fft_n)       */
  int32_t spec_pitch;              /* complex elements per half-spectrum row      */
  int32_t n_shells;
  int32_t max_order;
  int32_t max_offset[3];           /* max |m_a| over all shells                  */
  int64_t shell_size[CK_MAX_SHELLS];/* |O_s|, lattice offsets per shell          */
  int64_t n_multisets[CK_MAX_ORDER + 1]; /* C(N_s + n - 2, n - 1) for n = 2..5     */
  size_t workspace_bytes;
  int64_t bank_stride;             /* floats between shells in the W / B bank   */
  int32_t fused;                   /* 1: the last inverse FFT pass and the sums
                                      run as one kernel and no bank is kept
                                      (CK_PREC_SPLIT_TF32, n <= 3, <= 16 shells) */
  int32_t fft_n[3];                /* the transformed grid: n, or padded         */
} ck_plan_info;

/* Outputs of ck_compute.  For order n (index n = 2..5), xi[n], num[n] and
 * den[n] each point to a dense symmetric row-major [N_s]^(n-1) FP64 tensor
 * (host or device) or are NULL to skip.  num = sum_r N prod W_{s_i},
 * den = sum_r Rt prod B_{s_i}, xi = num / den (Eq. 11; NaN where den <= 0).
 * dropped (host or device, int64[2], may be NULL) receives the numbers of
 * data and random points that fell outside a non-periodic grid. */
typedef struct ck_outputs {
  double* xi[CK_MAX_ORDER + 1];
  double* num[CK_MAX_ORDER + 1];
  double* den[CK_MAX_ORDER + 1];
  int64_t* dropped;
} ck_outputs;

/* Workspace bytes ck_plan_create needs for these arguments (host only; no
 * CUDA call).  Returns CK_ERR_ARG / CK_ERR_UNSUPPORTED / CK_ERR_EMPTY_SHELL /
 * CK_ERR_KERNEL_TOO_LARGE exactly as ck_plan_create would. */
ck_status ck_plan_workspace_size(const ck_grid* grid, const ck_shells* shells,
                                 int32_t max_order, int32_t precision, size_t* bytes);

/* Build a plan: validate the arguments (before any CUDA call), build each
 * shell's offset list (Sec. 2.3), and compute every kernel spectrum
 * K^_s = DFT(K_s) / N_c on the device once (real and even, stored as an
 * octant).  `workspace` (device, >= ck_plan_workspace_size bytes, 256-byte
 * aligned) is borrowed for the plan's lifetime; NULL makes the plan allocate
 * and own it.  max_order in 2..5.  On error *out is NULL. */
ck_status ck_plan_create(const ck_grid* grid, const ck_shells* shells, int32_t max_order,
                         int32_t precision, void* workspace, size_t workspace_bytes,
                         void* stream, ck_plan** out);

/* Release the plan (synchronises its last stream; frees owned memory). */
ck_status ck_plan_destroy(ck_plan* plan);

ck_status ck_plan_get_info(const ck_plan* plan, ck_plan_info* info);

/* Grid the random catalog R (Sec. 2.2) and cache what depends on it alone:
 * the counts R, and the raw denominators den_raw_n = sum_r R prod (R***K_s)
 * (Eq. 10 with R unnormalised); ck_compute scales them by alpha^n, since
 * Rt = alpha R and B_s = alpha (R***K_s).  x, y, z: float32 positions, host
 * or device, n >= 0 points. */
ck_status ck_set_randoms(ck_plan* plan, const float* x, const float* y, const float* z,
                         int64_t n, void* stream);

/* One catalog through the whole path: grid D (Sec. 2.2), alpha = sum D /
 * sum R, N = D - alpha R (Eq. 8), W_s = N***K_s for every shell by FFT
 * (Eq. 9), the product sums num_n over all multisets of the orders in
 * order_mask (bit n set -> order n, 2..max_order; Eq. 11), den_n =
 * alpha^n den_raw_n, xi_n = num_n / den_n.  Needs ck_set_randoms first. */
ck_status ck_compute(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n,
                     int32_t order_mask, const ck_outputs* out, void* stream);

/* Weighted histograms (Sec. 2.2: "weighted count of tracers"; Sec. 3: the
 * survey's systematic and FKP weights): as ck_set_randoms / ck_compute, with
 * a float32 weight per point (w, in the same memory space as the positions).
 * A cell holds the sum of its points' weights: each weight is rounded to the
 * nearest multiple of 2^-32 (ties to even) and summed exactly in 64-bit
 * integers, so the sums do not depend on the order of addition; the cell
 * value is that sum rounded to float32.  alpha is the ratio of the exact
 * weight totals.  A point with a non-finite weight is dropped and counted.
 * Weighted and unweighted fields may be mixed (weighted data over unweighted
 * randoms and so on); ck_get_grids returns, for a weighted field, the float32
 * bit patterns of its cells. */
ck_status ck_set_randoms_weighted(ck_plan* plan, const float* x, const float* y, const float* z, const float* w,
                                  int64_t n, void* stream);
ck_status ck_compute_weighted(ck_plan* plan, const float* x, const float* y, const float* z, const float* w,
                              int64_t n, int32_t order_mask, const ck_outputs* out, void* stream);

/* --- survey input (Sec. 2.2) -------------------------------------------------- */

/* The fiducial cosmology of Eq. 3: H0 in km/s/Mpc (100 gives distances in
 * h^-1 Mpc), the present-day densities O_M, O_k, O_L, the speed of light c in
 * km/s, and the largest redshift of the catalog (the range of the distance
 * table). */
typedef struct ck_cosmology {
  double h0;
  double omega_m;
  double omega_k;
  double omega_l;
  double c;
  double z_max;
} ck_cosmology;

/* Sky coordinates to the grid's Cartesian frame: r = r(z) of Eq. 3,
 * r(z) = (c / H0) int_0^z dz' / sqrt(O_M (1+z')^3 + O_k (1+z')^2 + O_L),
 * evaluated on the device (a table of 4097 nodes on [0, z_max], 8-point
 * Gauss-Legendre quadrature per interval, cubic Hermite interpolation:
 * error below 1e-12 of r), then Eqs. 4-6: X = r cos(dec) cos(ra),
 * Y = r cos(dec) sin(ra), Z = r sin(dec), angles in degrees.  All six arrays
 * are device float32 of n entries (CK_ERR_BAD_POINTER otherwise); a redshift
 * outside [0, z_max] or a non-finite input gives NaN coordinates, which
 * gridding drops and counts.  CK_ERR_ARG for a non-finite or non-positive
 * h0, c or z_max, or E^2 <= 0 somewhere on [0, z_max].  Stream-ordered; the
 * distance table is a stream-ordered allocation freed after use. */
ck_status ck_sky_to_cartesian(const ck_cosmology* cosmo, const float* ra_deg, const float* dec_deg,
                              const float* redshift, int64_t n, float* x, float* y, float* z, void* stream);

/* A factorised selection (Sec. 2.2, Eq. 7): the angular density P_ang per
 * steradian on an equiangular grid of n_dec declination rows (row j covers
 * dec in [-90 + 180 j / n_dec, -90 + 180 (j+1) / n_dec) degrees) by n_ra
 * right-ascension columns (column i: ra in [360 i / n_ra, 360 (i+1) / n_ra)),
 * row-major with declination slowest; the redshift density P_z per unit z in
 * n_z equal bins of [z_lo, z_hi); N_tot the number of tracers.  Both tables
 * in HOST memory (copied at the call), entries finite and >= 0. */
typedef struct ck_selection {
  double n_tot;
  const double* p_ang;
  int32_t n_ra;
  int32_t n_dec;
  const double* p_z;
  int32_t n_z;
  int32_t pad;
  double z_lo;
  double z_hi;
} ck_selection;

/* The randoms field from the factorised selection instead of a random
 * catalog (Eq. 7): at every cell centre (X, Y, Z) of the plan's box, with
 * r = |(X, Y, Z)|, z = z(r) the inverse of Eq. 3 (the distance table of
 * ck_sky_to_cartesian, inverted per cell by Newton steps on its cubic
 * Hermite interpolant), ra = atan2(Y, X) in [0, 360), dec = asin(Z / r),
 *   R = N_tot P_ang(ra, dec) P_z(z) (dz/dr) g^3 / r^2,  dz/dr = H0 E(z) / c,
 * the cell's expected count (g^3 over the spherical volume element
 * r^2 dr dOmega, dr = dz c / (H0 E)), and R = 0 where z is outside
 * [z_lo, z_hi), r = 0 or r > r(z_max).  Every bin decision (and r against
 * r(z_max)) is that of an FP64 evaluation: cells clear of every edge by a
 * margin above the float32 error bound are evaluated in float32 (within
 * 8e-7 relative of the FP64 value), the others in FP64.  The cells are
 * stored as float32 (ck_get_grids returns their bits, as for weighted
 * fields), the field's total is their FP64 sum in a fixed order (the same
 * on every run), and
 * alpha = (data total) / (that total) as for any randoms field, so the xi
 * do not depend on N_tot.  Then the denominators of every order, as
 * ck_set_randoms.  Errors: CK_ERR_BAD_POINTER for NULL arguments or device
 * tables; CK_ERR_ARG for a cosmology ck_sky_to_cartesian rejects, table
 * sizes < 1 or > 2^20, n_ra * n_dec > 2^26, non-finite or negative entries or
 * N_tot, z_lo < 0 or z_hi <= z_lo; a field with no nonzero cell makes the
 * next ck_compute report CK_ERR_EMPTY_CATALOG.  On an argument error the
 * plan's previous randoms are kept.  Stream-ordered; scratch is a
 * stream-ordered allocation freed after use. */
ck_status ck_set_randoms_factorised(ck_plan* plan, const ck_cosmology* cosmo, const ck_selection* sel,
                                    void* stream);

/* The equidistant n-point functions alone (Sec. 2.6, Eq. 14): the same path
 * as ck_compute up to W_s, then for every shell s and requested order n only
 * the diagonal multiset (s, .., s):
 *   num_n[s] = sum_r W0 W_s^(n-1),  den_n[s] = alpha^n den_raw_n(s, .., s),
 *   xi_n[s] = num_n[s] / den_n[s],
 * in one pass over the bank, O(N_c N_s) instead of every multiset.  Plans
 * with the fused order-2/3 pass (no bank) take the diagonal entries of their
 * full sums.  Outputs (ck_outputs): xi[n], num[n], den[n] each hold N_s
 * doubles (host or device, caller-owned, NULL = skip), shell s at index s;
 * dropped as for ck_compute.  Same arguments and errors as ck_compute;
 * results are the diagonal entries of ck_compute's (equal to rounding of the
 * summation order).  Needs ck_set_randoms or ck_set_randoms_diagonal
 * first. */
ck_status ck_compute_diagonal(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n,
                              int32_t order_mask, const ck_outputs* out, void* stream);

/* ck_set_randoms for the diagonal alone: grid R and keep only the raw
 * denominators of the (s, .., s) multisets, from one pass over the random
 * field's bank (O(N_c N_s)); plans with the fused order-2/3 pass sum every
 * multiset as ck_set_randoms does.  Afterwards ck_compute_diagonal works;
 * ck_compute returns CK_ERR_NO_RANDOMS (unless every multiset was summed)
 * until ck_set_randoms is called. */
ck_status ck_set_randoms_diagonal(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n,
                                  void* stream);

/* --- fields on the grid and per-cell maps (Secs. 2.7, 2.8, 4.2) ----------------
 * Fields are float32 in the box's layout: n[2] x n[1] x n[0], x fastest (the
 * caller's box; padded plans place it in the corner of their transform
 * grid), each in device or host memory (host fields are staged through
 * plan scratch).  Values must be finite.  The randoms set on the plan stay
 * valid: a catalog's ck_compute may follow.  The data count grid
 * (ck_get_grids) is not defined afterwards.  On a non-periodic box plan the nonzero cells plus the
 * kernels' reach must fit the box (CK_ERR_GUARD_BAND otherwise, as for
 * catalogs); padded plans have no such limit. */

/* Continuous matter distribution (Sec. 2.7, Eqs. 15-17): the over-density
 * delta = (d - r) / r where r > 0, 0 where r <= 0 (outside the survey); r
 * NULL: d is delta itself.  W_0 = delta, W_s = delta *** K_s and
 *   xi_n(s_1..s_{n-1}) = sum_r W_0 W_s1 .. W_s(n-1)   (no denominator).
 * Outputs as ck_compute: xi[n] and num[n] receive the sums (dense symmetric
 * tensors), den[n] receives 1.0, dropped[0] receives 0 (dropped[1] keeps the
 * last randoms' count).  Needs no randoms.
 * Errors: CK_ERR_BAD_POINTER (plan or d NULL), CK_ERR_ARG (order mask), the
 * guard band as above. */
ck_status ck_compute_continuous(ck_plan* plan, const float* d, const float* r, int32_t order_mask,
                                const ck_outputs* out, void* stream);

/* Cross-correlation of two maps (Sec. 2.8): W_0 = f0, W_s = f1 *** K_s and
 * the same sums, sum_r f0 (f1***K_s1) .. (f1***K_s(n-1)); order 2 is Eq. 17
 * for two tracers.  Outputs, errors and field rules as
 * ck_compute_continuous; both fields required. */
ck_status ck_compute_cross(ck_plan* plan, const float* f0, const float* f1, int32_t order_mask,
                           const ck_outputs* out, void* stream);

/* The per-cell map W_0 W_s / <B_0 B_s> of shell `shell` (Sec. 4.2), for the
 * catalog of the last ck_compute (or ck_compute_weighted): W_0 = N,
 * W_s = N***K_s, and <B_0 B_s> = alpha^2 den_raw_2(s) / N_box, the average of
 * the random field's order-2 terms over the box's N_box cells.  map: float
 * [N_box] in box layout, device or host (host: synchronous, through the
 * data count buffer, which is then not defined).  Fused plans
 * recompute W_s from the resident spectrum first.  Errors:
 * CK_ERR_BAD_POINTER, CK_ERR_ARG (shell out of range, or the last call was
 * not a catalog's ck_compute), CK_ERR_NO_RANDOMS, CK_ERR_ZERO_DENOM (the
 * average is not positive: the map is NaN). */
ck_status ck_product_map(ck_plan* plan, int32_t shell, float* map, void* stream);

/* --- batched form --------------------------------------------------------------
 * Many catalogs over one or more plans (grid classes), each plan's randoms set
 * once with ck_set_randoms.  Catalog i is computed on plans[cats[i].plan] and
 * its outputs go to out[i] (as for ck_compute; out may be NULL).  On first use
 * of a (plan, order_mask) pair the plan's compute sequence for one catalog
 * (gridding through the normalised xi) is captured into a CUDA graph, on an
 * internal stream, after any synchronous preparation; every catalog then costs
 * one small descriptor kernel, one graph launch and its output copies.  A
 * plan's catalogs run in order; with catalogs on several plans, each plan's
 * run on a stream of the plan's own, forked from `stream` and joined back to
 * it, so that grid classes overlap (plans share no buffers).  The work is
 * ordered after earlier work on `stream`, and later work on `stream` after
 * it.  Positions must be device pointers (CK_ERR_BAD_POINTER
 * otherwise); results are the same as ck_compute's.  Device statuses are read
 * (and the stream synchronised) only if some output is in host memory. */
typedef struct ck_catalog {
  const float* x;
  const float* y;
  const float* z;
  int64_t n;
  int32_t plan;  /* index into `plans` */
} ck_catalog;

ck_status ck_batch_compute(ck_plan* const* plans, int32_t n_plans, const ck_catalog* cats, int32_t n_cats,
                           int32_t order_mask, const ck_outputs* out, void* stream);

/* Region of a catalog decomposed into slabs along z (Sec. 4: regions are
 * combined by adding the numerators and the denominators of Eq. 11 before
 * dividing, Eq. 19).  After this call the plan's sums run over the cells of
 * the box planes z_begin <= z < z_end only (the owned planes): the whole
 * box is still gridded and convolved, so planes outside the region act as
 * the halo that the kernels reach into, and only W_0 = N (and B_0 = Rt) is
 * restricted to the region.  alpha > 0 replaces sum D / sum R in
 * N = D - alpha R and Rt = alpha R, since every region of one catalog needs
 * the alpha of the whole catalog; 0 keeps the plan's own ratio.  With a box
 * of owned planes plus halos at least max_offset[2] planes deep (clipped at
 * the catalog's faces) on a CK_GRID_PADDED plan (zero outside the box), the
 * regions' num and den add up to the undivided catalog's.  Applies to
 * ck_set_randoms, ck_compute and their weighted forms; call ck_set_randoms
 * again afterwards (the cached denominators are dropped, and so are the
 * captured graphs of ck_batch_compute).  z_begin = 0, z_end = n[2],
 * alpha = 0 restores the whole box.  CK_ERR_ARG for an empty or
 * out-of-box range or a negative or non-finite alpha.  Host only. */
ck_status ck_plan_set_region(ck_plan* plan, int32_t z_begin, int32_t z_end, double alpha);

/* Autotuner (the batched and survey forms pick their transform and
 * contraction shapes per plan).  Times, on the plan's own buffers, the
 * candidates of each launch-shape choice that has more than one -- the z
 * step of the convolutions by the shells' short filters or by the forward
 * and K^ z passes (whichever gives the faster forward transform plus
 * inverse z and y passes), 8 or 16
 * columns per tile of the single-field 512-point strided passes, of the K^ z
 * pass and of the multi-shell inverse y pass (the latter two together), and
 * for the split tensor-core forms that keep a bank the widest tile stacked
 * (0, 32 or 64 columns: B's hi and lo side by side in one MMA, two MMAs per
 * k-step instead of three, which also adds the lo*lo term), 1, 2 or 3
 * contraction CTAs per SM, and whether the thin tiles run on a second
 * stream beside the tensor-core kernel -- each candidate once untimed and
 * five times between CUDA events, and keeps the one with the fastest run.  The tile
 * widths change launch shapes only: transforms are bit-identical, and the
 * contraction's sums differ by the order of their partial sums (and, for a
 * stacked tile, by its lo*lo term, below 2^-21 relative); the two z routes
 * give W_s that agree to FP32 rounding.  Needs a resident
 * field: the field, spectrum and bank that the last ck_set_randoms or
 * compute left are the inputs it times, and they are left as they were
 * (the spectrum of the same field, in either route's form)
 * (CK_ERR_NO_RANDOMS before either, and after ck_plan_set_region until the
 * next such call).  Captured graphs of ck_batch_compute are dropped.
 * Synchronises the stream. */
ck_status ck_plan_autotune(ck_plan* plan, void* stream);

/* The plan's current choices: out[0] columns per tile of the single-field
 * strided passes, out[1] of the K^ z pass, out[2] of the multi-shell inverse
 * y pass, out[3] contraction CTAs per SM, out[4] the widest stacked
 * contraction tile (columns; 0: none), out[5] 1 when thin tiles overlap
 * the tensor-core kernel, out[6] 1 when the convolutions take the z step
 * by the shells' short filters (plans whose shells reach at most 31 planes
 * in z; 0: the forward z pass and the K^ z pass), out[7] 1 once
 * ck_plan_autotune has run (else the defaults: 8, 8, 8, 2, 32, 1, 1 where
 * the plan has the filters). */
ck_status ck_plan_get_tuning(const ck_plan* plan, int32_t* out);

/* Set the choices by hand (in[0..6] as ck_plan_get_tuning's out[0..6]:
 * 8 or 16 columns, 1..3 CTAs per SM, 0..128 stacked columns, 0 or 1, 0 or
 * 1 (a plan without the filters keeps the transform route); CK_ERR_ARG
 * otherwise).  Host only; drops captured graphs and contraction plans. */
ck_status ck_plan_set_tuning(ck_plan* plan, const int32_t* in);

/* Synchronise `stream` and return (and clear) the plan's device status. */
ck_status ck_plan_status(ck_plan* plan, void* stream);

/* --- stage access (parity tests and diagnostics) ---------------------------- */

/* Copy the last data / random count grids (uint32 [N_c], device or host; either
 * may be NULL). */
ck_status ck_get_grids(ck_plan* plan, uint32_t* d_counts, uint32_t* r_counts, void* stream);

/* Copy a real field: which = 0 -> N of the last ck_compute (or the loaded
 * field of the last ck_compute_continuous / ck_compute_cross: delta, or f1),
 * which = 1 -> R (as float) of the last ck_set_randoms ... valid until the
 * next call that overwrites it (float [N_c], device or host). */
ck_status ck_get_field(ck_plan* plan, int32_t which, float* out, void* stream);

/* Copy shell `shell` of the convolution of the field whose spectrum is
 * resident: W_s = N***K_s after ck_compute, R***K_s after ck_set_randoms
 * (float [N_c], device or host).  CK_PREC_SPLIT_TF32 plans fuse the last
 * inverse pass with the sums and keep no bank; for them this call recomputes
 * the shell from the resident spectrum (one inverse transform on the
 * stream, overwriting internal scratch only). */
ck_status ck_get_bank(ck_plan* plan, int32_t shell, float* out, void* stream);

/* Copy the octant of K^_s = DFT(K_s) / N_c: float
 * [n[2]/2+1][n[1]/2+1][n[0]/2+1], device or host. */
ck_status ck_get_kernel_spectrum(ck_plan* plan, int32_t shell, float* out, void* stream);

/* Forward real-to-complex 3D DFT of a real field (device float [N_c]) into a
 * half spectrum (device float2 [n[2]][n[1]][spec_pitch]); unnormalised,
 * exponent sign -1.  Both pointers 16-byte aligned. */
ck_status ck_fft_r2c(ck_plan* plan, const float* in, void* out_spec, void* stream);

/* Inverse complex-to-real 3D DFT (exponent sign +1, unnormalised) of a half
 * spectrum (device, not modified) into a real field (device float [N_c]).
 * Both pointers 16-byte aligned; uses the plan's scratch spectra. */
ck_status ck_fft_c2r(ck_plan* plan, const void* in_spec, float* out, void* stream);

/* The summation stage alone (Sec. 2.5): for every order n in order_mask and
 * every multiset s_1 <= .. <= s_{n-1} (lexicographic order),
 * sums[n][j] = sum_r w0[r] prod_i bank[s_i * bank_stride + r].  w0: device
 * float [N_c]; bank: device float [N_s][bank_stride], bank_stride >= N_c and a
 * multiple of 4; sums[n]: device double [C(N_s + n - 2, n - 1)] or NULL. */
ck_status ck_contract(ck_plan* plan, const float* w0, const float* bank, int64_t bank_stride,
                      int32_t order_mask, double* const* sums, void* stream);

/* No-allocation variant of ck_contract (the paper has no counterpart): the
 * same summation (sums[n][j] = sum_r w0[r] prod_i bank[s_i * bank_stride + r]
 * over the multisets of order n in lexicographic order), for callers that
 * cannot allocate device memory -- a caller running inside another
 * framework's memory pool or a captured allocation-free region, or one that
 * must not grow its footprint after start-up.  It needs no plan: its scratch
 * (per-CTA partial sums and a status word, about 0.6 MB) is a fixed
 * file-scope device array that every GPU loading this library holds until
 * the process exits; it calls no allocator.  Limits: n_shells <= 16 with
 * orders <= 3, or n_shells <= 5 with orders <= 5 (otherwise
 * CK_ERR_UNSUPPORTED); at most 512 CTAs.  w0, bank: device float, 16-byte
 * aligned, n_cells cells each, bank_stride >= n_cells and a multiple of 4;
 * sums[n]: device double [C(n_shells + n - 2, n - 1)] or NULL.  The first
 * call on a device looks up the scratch address (cudaGetSymbolAddress) with
 * that device current, so make that first call before any stream capture.
 * Every call shares the one array: calls that overlap on the GPU (other
 * streams or threads) race and must be serialised by the caller.  If a
 * bounded device wait gives up, the outputs are NaN. */
ck_status ck_contract_static(const float* w0, const float* bank, int64_t bank_stride, int64_t n_cells,
                             int32_t n_shells, int32_t order_mask, double* const* sums, void* stream);

/* Test hook for the failure path of the bounded device waits (the paper has
 * no counterpart).  ns > 0: on the current device, every consumer warp of
 * the summation's register kernel (used by ck_contract for plain plans and
 * by ck_contract_static) first waits, with a limit of ns nanoseconds, on an
 * mbarrier that nothing arrives at.  The wait runs out, so each launch
 * records CK_ERR_TIMEOUT (in the plan's status word; ck_contract_static
 * returns NaN sums instead), consumes no staged chunk, waits with the
 * default limit (2 s) for the copies it has issued, and returns: no fault,
 * no hang, and the context stays usable.  ns <= 0 restores normal
 * operation.  Synchronous (cudaMemcpyToSymbol). */
ck_status ck_debug_force_timeout(int64_t ns);

/* --- per-stage device timing --------------------------------------------------
 * When enabled, the library records a CUDA event pair on the caller's stream
 * around every kernel it launches, grouped by stage, together with the
 * algorithmic bytes that launch must move (inputs read once + outputs written
 * once).  ck_profile_enable resets the accumulators; ck_profile_read
 * synchronises each recorded event and returns the totals. */
/* Stages 0..14: grid_points, prepare_field, fft_x_r2c, fft_y_fwd, fft_z_fwd,
 * fft_z_inv_mul, fft_y_inv, fft_x_c2r, contract, reduce, finalize,
 * x_c2r_contract (the inverse x pass fused with the order-2/3 sums), other,
 * selection_field (the factorised randoms of Eq. 7; bytes = the cells
 * written), z_conv (the z step of the convolution by the shells' short
 * filters, in place of fft_z_fwd and fft_z_inv_mul). */
#define CK_STAGES 15
typedef struct ck_stage_times {
  double ms[CK_STAGES];       /* summed event time of the stage's launches   */
  int64_t launches[CK_STAGES];
  double bytes[CK_STAGES];    /* summed algorithmic bytes of those launches  */
} ck_stage_times;

ck_status ck_profile_enable(ck_plan* plan, int32_t enable);
ck_status ck_profile_read(ck_plan* plan, ck_stage_times* out);
/* Name of stage i (0 <= i < CK_STAGES), or NULL. */
const char* ck_stage_name(int32_t stage);

const char* ck_status_string(ck_status status);
int32_t ck_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CONKER_H */
