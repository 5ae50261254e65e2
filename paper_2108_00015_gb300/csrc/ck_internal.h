// ck_internal.h -- private declarations shared by the library's translation
// units (plan layout, launch helpers).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "conker.h"

namespace ck {

// Device-side state of a plan: point counters, occupied-cell bounding boxes,
// alpha and the status word.  Index 0 = data catalog, 1 = randoms.
// A catalog's device positions, read by the gridding kernel of a captured graph.
struct CatalogRef {
  const float* x;
  const float* y;
  const float* z;
  int64_t n;
};

struct DevState {
  unsigned long long kept[2];
  long long wsum[2];  // weighted fields: the kept points' weights, in units of 2^-32
  int weighted[2];    // 1: cells hold float32 weight sums, total wsum; 2: float32 cells, total fsum
  unsigned long long dropped[2];
  int bbox_min[2][3];
  int bbox_max[2][3];
  int status;
  int pad;
  double alpha;
  double fsum[2];     // fields computed in place (weighted == 2): the FP64 total of the cells
  // planes z0..z1 outside which the field buffer is zero (field_known: the
  // record holds; 0, as at plan creation or after a field was loaded: unknown)
  int field_known;
  int field_z0, field_z1;
  // count buffer k is zero outside the planes of bbox[k] (nonzero: the
  // record holds; 0, as at plan creation or after the buffer served as
  // staging: unknown)
  int counts_known[2];
  int pad2;
};

constexpr int kMaxStages = 8;

// Radix decomposition of one transform length: radices 5 and 3 first, then
// the power of two as radix 8 and 4 (radix 2 only when 2 is the whole power
// of two), or a single radix 1 for length 1.
struct RPlan {
  int nst;
  int r[kMaxStages];
};

__host__ __device__ constexpr RPlan rplan(int n) {
  RPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}};
  int m = n, p2 = 0;
  while (m > 0 && m % 2 == 0) { m /= 2; ++p2; }
  while (m > 1 && m % 5 == 0 && p.nst < kMaxStages) { p.r[p.nst++] = 5; m /= 5; }
  while (m > 1 && m % 3 == 0 && p.nst < kMaxStages) { p.r[p.nst++] = 3; m /= 3; }
  if (m != 1) return RPlan{-1, {0, 0, 0, 0, 0, 0, 0, 0}};
  if (p2 >= 4 && p2 % 3 == 1) { p.r[p.nst++] = 4; p.r[p.nst++] = 4; p2 -= 4; }
  while (p2 >= 3 && p.nst < kMaxStages) { p.r[p.nst++] = 8; p2 -= 3; }
  if (p2 == 2) p.r[p.nst++] = 4;
  if (p2 == 1) p.r[p.nst++] = 2;
  if (p.nst == 0) p.r[p.nst++] = 1;
  return p;
}

// Radix decomposition of one transform length (runtime copy of rplan).
struct FftLen {
  int n = 0;
  int nst = 0;
  int radix[kMaxStages] = {0};
};

// Operand descriptors of the blocked contraction: row p of A is
// w0 * W[i] * W[j], column q of B is W[k] * W[l] (an index of -1 = factor 1).
struct ContractPlan {
  int order_mask = 0;
  bool use_reg = false;     // register-accumulator kernel (few outputs)
  bool use_tc = false;      // blocked product on the tensor cores (split-TF32 / BF16 / FP16, tcgen05)
  int um_kind = 0;          // tcgen05 operand kind: 0 TF32, 1 BF16, 2 FP16
  int um_tn = 0;            // tcgen05 tiles: 128 rows x at most um_tn columns
  int um_ntc = 0;           // tiles 0 .. um_ntc - 1 on the tensor cores, the rest thin (CUDA cores)
  int um_thin_rmax = 0;     // the most live rows of a thin tile
  int64_t um_cps = 0;       // tcgen05: cells per split
  int reg_maxn = 0;         // orders 2..reg_maxn computed by that kernel
  int n_out_reg = 0;        // outputs of the register kernel
  int rows = 0, cols = 0;   // blocked kernel: operand rows / columns
  int n_tiles = 0;          // blocked kernel: active 64 x 64 output tiles
  int splits = 0;           // CTAs along the cell dimension
  int ctas = 0;             // register kernel: CTAs
  int64_t chunks_per_cta = 0;
  // device tables (inside the workspace)
  int2* d_rowdesc = nullptr;
  int2* d_coldesc = nullptr;
  int2* d_tiles = nullptr;   // (m0, n0) per active tile
  int4* d_um_tiles = nullptr;  // tcgen05: (m0, column-list offset, MMA N, columns) per tile
  int* d_um_cols = nullptr;    // tcgen05: the tiles' column lists
  int* d_slot = nullptr;     // [n_tiles][64][64] -> output slot or -1
  size_t partial_doubles = 0;
};

// Per-stage event timing (ck_profile_enable / ck_profile_read).
enum Stage {
  ST_GRID = 0, ST_PREP, ST_FFT_X_R2C, ST_FFT_Y_FWD, ST_FFT_Z_FWD, ST_FFT_Z_INV_MUL, ST_FFT_Y_INV,
  ST_FFT_X_C2R, ST_CONTRACT, ST_REDUCE, ST_FINALIZE, ST_X_C2R_CONTRACT, ST_OTHER, ST_SELECTION, ST_Z_CONV
};

struct Profiler {
  bool on = false;
  // bytes of a launch: `bytes`, plus per_row x (rows) + per_plane x (planes)
  // of the support box copied to the pinned slot of the record (boxed)
  struct Rec { int stage; double bytes; cudaEvent_t a, b; bool boxed; double per_row, per_plane; };
  std::vector<Rec> recs;      // event pool; recs[0..used) are pending
  size_t used = 0;
  double ms[CK_STAGES] = {0};
  int64_t launches[CK_STAGES] = {0};
  double bytes[CK_STAGES] = {0};
  int64_t dropped = 0;        // launches not recorded (pool exhausted)
  int* pin = nullptr;         // page-locked: 6 ints per record (support boxes)
};

// Choices the autotuner makes per plan (ck_plan_autotune); the defaults are
// the measured best on the survey workloads.
struct Tuning {
  int fwd_cols = 8;        // columns per tile of the single-field 512-point strided passes
  int zreg_cols = 8;       // of the K^ z pass (every shell)
  int yinv_cols = 8;       // of the multi-shell inverse y pass
  int tc_ctas_per_sm = 2;  // tensor-core contraction: CTAs per SM the splits aim at
  int tc_stack_cols = 32;  // tensor-core tiles of at most this many columns are stacked (0: none)
  int tc_thin_overlap = 1; // 1: thin tiles on a second stream beside the tensor-core kernel
  int z_direct = 1;        // 1: the z step of the convolution by its short filter (where the plan has one)
  bool tuned = false;
};

struct Plan {
  ck_grid grid{};
  int ns = 0;
  double width = 0;
  int rule = 0;
  int max_order = 0;
  int precision = 0;
  std::vector<double> radius;
  std::vector<std::vector<int>> offsets;  // per shell: flattened (mx, my, mz)
  int maxoff[3] = {0, 0, 0};
  int box_n[3] = {0, 0, 0};  // the caller's box (points outside are dropped); grid.n is the transformed grid
  int64_t nc = 0;
  int px = 0;               // half-spectrum row pitch (complex elements)
  int64_t spec_elems = 0;   // n[2] * n[1] * px
  int64_t field_stride = 0; // floats reserved per real field (>= nc, multiple of 64)
  int oct[3] = {0, 0, 0};   // octant extents n/2 + 1
  int64_t oct_elems = 0;
  int64_t khat_stride = 0;  // floats per shell spectrum: octant rows padded to px (zeros beyond n[0]/2)
  int H = 0;                // max offset over all shells and axes
  // The z step by direct filtering (ck_zconv.cu): taps per column (0: the
  // plan has no table), groups of 4 shells, taps per group, the table
  float* kzt = nullptr;
  int kz_dz = 0;
  int kz_groups = 0;
  int kz_taps[CK_MAX_SHELLS] = {0};
  int64_t kz_group_stride = 0;  // floats per group of the table
  // the resident spectrum p.spec was left untransformed along z (the last
  // forward transform into it took the direct route), and the box (device)
  // outside whose planes its field vanishes (null: every plane transformed)
  mutable bool spec_direct = false;
  mutable const int* spec_in_box = nullptr;
  int64_t n_multisets[CK_MAX_ORDER + 1] = {0};
  int64_t multiset_base[CK_MAX_ORDER + 1] = {0};  // offset of order n in a packed array
  int64_t n_multiset_total = 0;
  int64_t dense_elems[CK_MAX_ORDER + 1] = {0};
  int64_t dense_base[CK_MAX_ORDER + 1] = {0};
  int64_t dense_total = 0;
  FftLen fx_half, fy, fz;   // x uses a half-length complex transform

  // workspace
  void* ws = nullptr;
  bool owns_ws = false;
  size_t ws_bytes = 0;
  uint32_t* counts[2] = {nullptr, nullptr};  // counts, or the float32 bits of weight sums (DevState::weighted)
  long long* wacc = nullptr;  // [nc] fixed-point weight sums of the field being gridded
  float* field = nullptr;
  float2* spec = nullptr;
  float2* tmp = nullptr;
  float* khat = nullptr;
  float* bank = nullptr;
  double* partials = nullptr;
  size_t partials_cap = 0;  // doubles
  float* staging = nullptr;
  int64_t staging_pts = 0;  // points per staging slot
  float* thr[3] = {nullptr, nullptr, nullptr};   // cell-edge thresholds, n+1 each
  float2* tw[3] = {nullptr, nullptr, nullptr};   // e^{-2 pi i t / n_a}, n_a each
  float2* twm = nullptr;  // e^{-2 pi i l2 m1 / 512} at [m1 * 32 + l2], m1 < 16, l2 < 32 (K^ z pass)
  float2* stw[3] = {nullptr, nullptr, nullptr};  // per-iteration twiddles of the y, z and half-x lengths
  DevState* dstate = nullptr;
  double* den_raw = nullptr;   // packed per order (multiset order)
  double* sums = nullptr;      // packed per order: num of the last compute
  double* dense = nullptr;     // 3 x dense_total: xi, num, den staging
  int* dense_map = nullptr;    // packed per order: dense index -> multiset rank
  int* host_status_pinned = nullptr;
  int* support = nullptr;      // [12] boxes of the cells where W_0 (0..5) and the field (6..11) may be nonzero
  unsigned* absmax = nullptr;  // [CK_MAX_SHELLS + 1] largest |W| per factor row (split-FP16 scales)

  ContractPlan cplan[1 << (CK_MAX_ORDER + 1)];
  bool cplan_ready[1 << (CK_MAX_ORDER + 1)] = {false};
  unsigned char* table_arena = nullptr;  // contraction tables
  size_t table_arena_cap = 0, table_arena_used = 0;

  mutable Profiler prof;

  // batched form: the catalog descriptor and one instantiated graph per order mask
  CatalogRef* dref = nullptr;
  cudaStream_t cap_stream = nullptr;
  // ck_batch_compute over several plans: this plan's catalogs run on its own
  // stream, forked from and joined to the caller's (fork, join events)
  cudaStream_t batch_stream = nullptr;
  cudaEvent_t batch_fork = nullptr, batch_join = nullptr;
  // the contraction's thin tiles beside its tensor-core kernel (tc_thin_overlap)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
  cudaGraphExec_t gexec[1 << (CK_MAX_ORDER + 1)] = {nullptr};

  bool have_randoms = false;       // den_raw holds every multiset of the plan's orders
  bool have_randoms_diag = false;  // den_raw holds at least the (s, .., s) multisets
  int bank_holds = -1;  // field whose spectrum is resident: 0 = data, 1 = randoms
  // Convolution and sums in one pass (FP32, <= 16 shells, orders <= 3): the
  // bank is not kept; `bank` holds one field, recomputed on request.
  bool fused = false;
  int bank_fields = 0;      // real fields reserved in `bank`
  int device = 0;
  int sm_count = 0;
  Tuning tune;
  // Region of a decomposed catalog (ck_plan_set_region): the sums run over
  // the box planes region_z0 <= z < region_z1 only; region_alpha > 0 is used
  // in place of sum D / sum R.
  int region_z0 = 0, region_z1 = 0;
  bool region = false;
  double region_alpha = 0.0;
};

// ---- host helpers (ck_plan.cu) ------------------------------------------------
ck_status validate_and_layout(const ck_grid* grid, const ck_shells* shells, int max_order,
                              int precision, Plan* p);
size_t workspace_bytes(const Plan& p);
size_t khat_scratch_doubles(const Plan& p);
bool factor_len(int n, FftLen* out);
ck_status cuda_status(cudaError_t e);
bool is_device_ptr(const void* p);  // device or managed memory
int64_t binom(int64_t n, int64_t k);

// Record the start / end of one launch of `stage` (no-ops unless enabled).
int prof_begin(const Plan& p, int stage, double bytes, cudaStream_t st);
// The same for a launch that visits the support box `box` (device): its
// bytes are counted when the times are read.
int prof_begin_box(const Plan& p, int stage, double bytes, double per_row, double per_plane, const int* box,
                   cudaStream_t st);
void prof_end(const Plan& p, int idx, cudaStream_t st);

struct ProfScope {
  const Plan& p;
  int idx;
  cudaStream_t st;
  ProfScope(const Plan& pl, int stage, double bytes, cudaStream_t s)
      : p(pl), idx(prof_begin(pl, stage, bytes, s)), st(s) {}
  ProfScope(const Plan& pl, int stage, double bytes, double per_row, double per_plane, const int* box,
            cudaStream_t s)
      : p(pl), idx(box ? prof_begin_box(pl, stage, bytes, per_row, per_plane, box, s) : prof_begin(pl, stage, bytes, s)),
        st(s) {}
  ~ProfScope() { prof_end(p, idx, st); }
};

// ---- launches (ck_grid.cu) ---------------------------------------------------
void launch_grid_points(const Plan& p, const float* x, const float* y, const float* z, int64_t n,
                        int which, cudaStream_t st);
void launch_set_catalog_ref(const Plan& p, const float* x, const float* y, const float* z, int64_t n,
                            cudaStream_t st);
void launch_grid_points_ref(const Plan& p, int which, cudaStream_t st);  // catalog from p.dref
// Zero count buffer `which` where it may be nonzero (the planes of the last
// histogram's box, or everywhere if unknown) and record it as known; then
// reset the field's state (kept, box) for a new histogram.
cudaError_t launch_clear_counts(const Plan& p, int which, cudaStream_t st);
void launch_prepare_data(const Plan& p, cudaStream_t st);     // alpha, N -> field, checks
void launch_prepare_randoms(const Plan& p, cudaStream_t st);  // R (float) -> field
// p.support = the box where W_0 may be nonzero: mode 0 data (D and R
// occupied), 1 randoms; clipped to the region's planes (support[0..5]),
// unclipped (support[6..11]); support[12..13]: the planes the field's
// preparation rewrites (the box's and those where the field may be nonzero
// from before), after which the field is zero outside the box's planes.
void launch_support_box(const Plan& p, int mode, cudaStream_t st);
// The factorised randoms field of Eq. 7 (ck_sky.cu): check_factorised
// validates the arguments; launch_factorised_randoms writes counts[1] (float
// bits) and the field's totals, after the caller has reset field 1.
ck_status check_factorised(const ck_cosmology* cosmo, const ck_selection* sel);
ck_status launch_factorised_randoms(Plan& p, const ck_cosmology* cosmo, const ck_selection* sel, cudaStream_t st);
// Weighted gridding into p.wacc (zeroed by the caller), then the cells of field `which`.
void launch_grid_points_weighted(const Plan& p, const float* x, const float* y, const float* z, const float* w,
                                 int64_t n, int which, cudaStream_t st);
void launch_weights_to_cells(const Plan& p, int which, cudaStream_t st);

// ---- launches (ck_fft.cu) ----------------------------------------------------
ck_status fft_init_attributes();
// box (device, may be null): the field is zero outside it, and the passes
// skip the rows and planes that hold only zeros (512-point y and z axes).
// conv: the spectrum is for the plan's convolutions (into p.spec), which
// leave out the z transform when the plan takes the direct z step
// (p.spec_direct records which form p.spec holds); otherwise a full 3D
// transform.
void launch_fft_forward(const Plan& p, const float* in, float2* spec, cudaStream_t st, const int* box = nullptr,
                        bool conv = false);
// Inverse transforms of nshells spectra (spec * K^_s for shells shell0 ..
// shell0 + nshells - 1, or spec alone when shell0 < 0) through scratch
// spectra tmp[s] into real fields out + s * out_stride.  With shell0 >= 0,
// spec is p.spec in the form p.spec_direct records.  box (device, may be
// null): only the planes z0..z1 of each field are written (the others keep
// what they held).
void launch_fft_inverse(const Plan& p, const float2* spec, int shell0, int nshells, float2* tmp, float* out,
                        int64_t out_stride, cudaStream_t st, const int* box = nullptr);
// Its first two passes alone: tmp[s] = (y, z inverse of spec * K^_s), rows of pitch px.
// box (device, may be null): only the planes z0..z1 of the output are
// needed, and of them, for fused plans, only the rows y0..y1.
void launch_inverse_zy(const Plan& p, const float2* spec, int shell0, int nshells, float2* tmp, cudaStream_t st,
                       const int* box = nullptr);
ck_status build_kernel_spectra(Plan& p, cudaStream_t st);

// ---- the direct z step (ck_zconv.cu) ------------------------------------------
constexpr int kZconvGroup = 4;               // shells per group of the table
void zconv_layout(Plan& p);                  // kz_dz, kz_groups, kz_taps, kz_group_stride
size_t zconv_table_bytes(const Plan& p);     // 0 without a table
// The table from the FP64 (x, y) cosine sums of build_kernel_spectra.
cudaError_t launch_zconv_table(const Plan& p, const double* A2, cudaStream_t st);
// out + (s - shell0) * out_stride = the z step of W_s for shells shell0 ..
// shell0 + nshells - 1 from spec (transformed along x and y).  in_box
// (device, may be null): spec vanishes outside its planes z = in_box[4] ..
// in_box[5], whatever the others hold; out_box (may be null): only its
// planes are written (null: every plane).
void launch_zconv(const Plan& p, const float2* spec, int shell0, int nshells, float2* out, int64_t out_stride,
                  const int* in_box, const int* out_box, cudaStream_t st);

// ---- fused inverse x pass + sums (ck_xc.cu) -----------------------------------
int xc_pad_shells(int ns);               // supported padded shell count, 0 if none
size_t xc_smem_bytes(int M, int ns_pad);  // shared memory of the fused kernel
// Inverse z, y passes and the fused x pass + order-2/3 sums of the resident
// spectrum p.spec with cell values w0; packed sums (orders <= max_order).
// box (device, may be null): W_0 vanishes outside it, so the passes visit
// only its rows and planes.
ck_status launch_convolve_contract(Plan& p, const float* w0, double* sums, cudaStream_t st, const int* box);

// ---- tcgen05 blocked product (ck_umma.cu) -------------------------------------
constexpr int kUmmaStacked = 1 << 16;
int umma_tile_rows();
int umma_tile_cols(int cols);
int64_t umma_cells_per_split(int64_t nc, int ntiles, int sm_count, int ctas_per_sm = 2);
// A tile is (first row, offset of its column list, MMA N <= tn, list length
// L, plus kUmmaStacked for a stacked tile).  A stacked tile puts the hi and
// lo parts of each B column side by side (columns q and N/2 + q, N = 2 x L
// rounded up to 16) and issues A_hi x B and A_lo x B per k-step, two MMAs
// instead of three; its partials hold both halves, which the reduction adds.
// Tensor-core tiles 0 .. ntc - 1 of ntiles (the partials are pitched by ntiles).
// kind: 0 split-TF32, 1 split-BF16, 2 split-FP16 (absmax: ns + 1 device
// words for the FP16 scales, filled here).
// box (device, may be null): only the planes z0..z1 of the support box are
// summed (plane cells each); splits share them out in whole 256-cell groups.
// min_smem: dynamic shared memory to request at least (0: what the tile
// shape needs); a larger request keeps one CTA per SM, leaving room beside it.
cudaError_t launch_umma(int tn, int kind, const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns,
                        const int2* rowdesc, int rows, const int2* coldesc, const int4* tiles, const int* collist,
                        int ntc, int ntiles, int splits, const int* box, int64_t plane, unsigned* absmax,
                        double* partials, int* status, cudaStream_t st, size_t min_smem = 0);
// Thin tiles (at most kThinMaxOut outputs, kThinMaxCols columns) t0 .. t0 + nthin - 1 on the CUDA
// cores in FP32, into the same partials layout (tile width tn).
constexpr int kThinMaxOut = 256;
constexpr int kThinMaxCols = 16;
size_t umma_thin_smem(int ns, int rmax);  // rmax: the most live rows of a thin tile
cudaError_t launch_umma_thin(const float* w0, const float* bank, int64_t bstride, int64_t nc, int ns, int rmax,
                             const int2* rowdesc, int rows, const int2* coldesc, const int4* tiles,
                             const int* collist, int t0, int nthin, int ntiles, int tn, int splits, const int* box,
                             int64_t plane, double* partials, cudaStream_t st);
cudaError_t launch_umma_reduce(const double* partials, int splits, int ntiles, int tn, const int4* tiles,
                               const int* collist, const int2* rowdesc, int rows, const int2* coldesc, int mask,
                               int ns, const int64_t* bases, double* out, cudaStream_t st);

// ---- launches (ck_contract.cu) -----------------------------------------------
ck_status contract_prepare(Plan& p, int order_mask);
// box (device, may be null): W_0 vanishes outside the support box, and
// only its planes are summed.
ck_status launch_contract(Plan& p, int order_mask, const float* w0, const float* bank,
                          int64_t bank_stride, double* sums_packed, cudaStream_t st, const int* box = nullptr);
// plain: field sums with no denominator (xi = num, den = 1)
void launch_finalize(const Plan& p, int order_mask, cudaStream_t st, bool plain = false);

// ---- fields on the grid and product maps (ck_fields.cu) -----------------------
// a (and b) in box layout -> out in the stored layout: a copy, or (delta)
// Eq. 15's (a - b) / b where b > 0, 0 elsewhere (b NULL: a itself); the
// nonzero cells' count and box go to field `which` of the plan state.
void launch_field_load(const Plan& p, const float* a, const float* b, bool delta, float* out, int which,
                       cudaStream_t st);
void launch_field_check(const Plan& p, cudaStream_t st);  // guard band over field 0's extent
// out (box layout) = w0 ws / <B_0 B_s>, <B_0 B_s> = alpha^2 den_raw_2(shell) / N_box
void launch_product_map(const Plan& p, const float* w0, const float* ws, int shell, float* out, cudaStream_t st);
// Eq. 14 for the orders in order_mask after the forward transform of the
// plan's field: num/den/xi of (s, .., s) for every shell into the first N_s
// entries of each order's dense outputs (ck_diag.cu).
ck_status launch_diagonal(Plan& p, int order_mask, cudaStream_t st);
// The random field's diagonal sums (s, .., s) into den_raw after its forward
// transform; *full is set when every multiset was summed (fused plans).
ck_status launch_diagonal_randoms(Plan& p, bool* full, cudaStream_t st);
// Rank of the non-decreasing shell sequence s[0..k-1] among all of its
// length over ns shells, in the packed (lexicographic) order.
int64_t host_multiset_rank(const int* s, int k, int ns);

}  // namespace ck
