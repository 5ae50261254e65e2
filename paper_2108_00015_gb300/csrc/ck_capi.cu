// ck_capi.cu -- the C ABI (conker.h): plan life cycle, the per-catalog
// pipeline (mapping -> FFT convolution -> summation -> xi) and stage access.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ck_device.cuh"
#include "ck_internal.h"

namespace ck {
int64_t host_multiset_rank(const int* s, int k, int ns);

int prof_begin(const Plan& p, int stage, double bytes, cudaStream_t st) {
  Profiler& f = p.prof;
  if (!f.on) return -1;
  if (f.used >= f.recs.size()) {
    ++f.dropped;
    return -1;
  }
  Profiler::Rec& r = f.recs[f.used];
  r.stage = stage;
  r.bytes = bytes;
  r.boxed = false;
  if (cudaEventRecord(r.a, st) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (int)f.used++;
}

int prof_begin_box(const Plan& p, int stage, double bytes, double per_row, double per_plane, const int* box,
                   cudaStream_t st) {
  const int idx = prof_begin(p, stage, bytes, st);
  if (idx < 0 || !p.prof.pin) return idx;
  Profiler::Rec& r = p.prof.recs[(size_t)idx];
  if (cudaMemcpyAsync(p.prof.pin + 6 * (size_t)idx, box, 6 * sizeof(int), cudaMemcpyDeviceToHost, st) ==
      cudaSuccess) {
    r.boxed = true;
    r.per_row = per_row;
    r.per_plane = per_plane;
  } else {
    cudaGetLastError();
  }
  return idx;
}

void prof_end(const Plan& p, int idx, cudaStream_t st) {
  if (idx < 0) return;
  if (cudaEventRecord(p.prof.recs[(size_t)idx].b, st) != cudaSuccess) cudaGetLastError();
}
}  // namespace ck

namespace {
constexpr size_t kProfPool = 16384;
const char* kStageNames[CK_STAGES] = {"grid_points", "prepare_field", "fft_x_r2c", "fft_y_fwd",
                                      "fft_z_fwd", "fft_z_inv_mul", "fft_y_inv", "fft_x_c2r",
                                      "contract", "reduce", "finalize", "x_c2r_contract", "other",
                                      "selection_field", "z_conv"};

void prof_collect(ck::Plan& p) {
  ck::Profiler& f = p.prof;
  for (size_t i = 0; i < f.used; ++i) {
    ck::Profiler::Rec& r = f.recs[i];
    float ms = 0.0f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      f.ms[r.stage] += ms;
      f.launches[r.stage] += 1;
      double b = r.bytes;
      if (r.boxed) {  // the support box this launch visited (copied before it ran)
        const int* bx = f.pin + 6 * i;
        const double ny = std::max(0, bx[3] - bx[2] + 1), nz = std::max(0, bx[5] - bx[4] + 1);
        b += r.per_row * ny * nz + r.per_plane * nz;
      }
      f.bytes[r.stage] += b;
    } else {
      cudaGetLastError();
    }
  }
  f.used = 0;
}

}  // namespace

// Device memory (or managed) vs host memory.
bool ck::is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

using namespace ck;

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define CK_TRY(expr)                                  \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_status(e_);    \
  } while (0)

#define CK_TRY_S(expr)                                \
  do {                                                \
    ck_status s_ = (expr);                            \
    if (s_ != CK_OK) return s_;                       \
  } while (0)

__global__ void reset_state_kernel(DevState* st, int which) {
  st->kept[which] = 0;
  st->wsum[which] = 0;
  st->weighted[which] = 0;
  st->fsum[which] = 0.0;
  st->dropped[which] = 0;
  for (int a = 0; a < 3; ++a) {
    st->bbox_min[which][a] = 0x7fffffff;
    st->bbox_max[which][a] = -0x7fffffff - 1;
  }
}

size_t al(size_t b) { return (b + 255) / 256 * 256; }

ck_status carve(Plan& p) {
  unsigned char* b = static_cast<unsigned char*>(p.ws);
  auto take = [&](size_t bytes) {
    unsigned char* r = b;
    b += al(bytes);
    return r;
  };
  p.counts[0] = reinterpret_cast<uint32_t*>(take((size_t)p.nc * 4));
  p.counts[1] = reinterpret_cast<uint32_t*>(take((size_t)p.nc * 4));
  p.field = reinterpret_cast<float*>(take((size_t)p.field_stride * 4));
  p.spec = reinterpret_cast<float2*>(take((size_t)p.spec_elems * 8));
  p.tmp = reinterpret_cast<float2*>(take((size_t)p.ns * p.spec_elems * 8));
  p.khat = reinterpret_cast<float*>(take((size_t)p.ns * p.khat_stride * 4));
  p.bank = reinterpret_cast<float*>(take(std::max((size_t)p.bank_fields * p.field_stride * 4, khat_scratch_doubles(p) * 8)));
  p.partials = reinterpret_cast<double*>(take(p.partials_cap * 8));
  p.staging = reinterpret_cast<float*>(take((size_t)2 * 4 * p.staging_pts * 4));
  p.wacc = reinterpret_cast<long long*>(take((size_t)p.nc * 8));
  for (int a = 0; a < 3; ++a) p.thr[a] = reinterpret_cast<float*>(take((size_t)(p.grid.n[a] + 1) * 4));
  for (int a = 0; a < 3; ++a) p.tw[a] = reinterpret_cast<float2*>(take((size_t)p.grid.n[a] * 8));
  for (int a = 0; a < 3; ++a) p.stw[a] = reinterpret_cast<float2*>(take((size_t)p.grid.n[a] * 8));
  p.twm = reinterpret_cast<float2*>(take((size_t)512 * 8));
  p.dstate = reinterpret_cast<DevState*>(take(sizeof(DevState)));
  p.dref = reinterpret_cast<CatalogRef*>(take(sizeof(CatalogRef)));
  p.den_raw = reinterpret_cast<double*>(take((size_t)std::max<int64_t>(p.n_multiset_total, 1) * 8));
  p.sums = reinterpret_cast<double*>(take((size_t)std::max<int64_t>(p.n_multiset_total, 1) * 8));
  p.dense = reinterpret_cast<double*>(take((size_t)3 * std::max<int64_t>(p.dense_total, 1) * 8));
  p.dense_map = reinterpret_cast<int*>(take((size_t)std::max<int64_t>(p.dense_total, 1) * 4));
  p.table_arena = take(p.table_arena_cap);
  p.support = reinterpret_cast<int*>(take(14 * 4));
  p.absmax = reinterpret_cast<unsigned*>(take((size_t)(CK_MAX_SHELLS + 1) * 4));
  p.kzt = p.kz_dz > 0 ? reinterpret_cast<float*>(take(zconv_table_bytes(p))) : nullptr;
  const size_t used = (size_t)(b - static_cast<unsigned char*>(p.ws));
  return used <= p.ws_bytes ? CK_OK : CK_ERR_OOM;
}

// Smallest float32 >= fl64(origin + fl64(k * cell)), k = 0..n.
void thresholds(double o, double g, int n, std::vector<float>& t) {
  t.resize((size_t)n + 1);
  for (int k = 0; k <= n; ++k) {
    volatile double prod = (double)k * g;
    const double e = o + prod;
    float f = (float)e;
    if ((double)f < e) f = nextafterf(f, INFINITY);
    t[(size_t)k] = f;
  }
}

// Per-iteration twiddles of a length-n transform: for iteration i (radix R,
// Ns = product of the earlier radices), entries k * (R - 1) + r - 1 hold
// e^{-2 pi i r k / (Ns R)}, k < Ns, 1 <= r < R.
void stage_twiddles(int n, std::vector<float2>& w) {
  const RPlan pl = rplan(n);
  w.clear();
  int ns = 1;
  for (int i = 0; i < pl.nst; ++i) {
    const int R = pl.r[i];
    for (int k = 0; k < ns; ++k)
      for (int r = 1; r < R; ++r) {
        const long long num = ((long long)r * k) % ((long long)ns * R);
        const double a = 2.0 * M_PI * (double)num / (double)(ns * R);
        w.push_back(make_float2((float)cos(a), (float)-sin(a)));
      }
    ns *= R;
  }
  if (w.empty()) w.push_back(make_float2(1.f, 0.f));
}

void twiddles(int n, std::vector<float2>& w) {
  w.resize((size_t)n);
  for (int t = 0; t < n; ++t) {
    const double a = 2.0 * M_PI * (double)t / (double)n;
    w[(size_t)t] = make_float2((float)cos(a), (float)-sin(a));
  }
}

ck_status upload_tables(Plan& p, cudaStream_t st) {
  for (int a = 0; a < 3; ++a) {
    std::vector<float> t;
    thresholds(p.grid.origin[a], p.grid.cell, p.box_n[a], t);  // cells of the box
    CK_TRY(cudaMemcpy(p.thr[a], t.data(), t.size() * 4, cudaMemcpyHostToDevice));
    std::vector<float2> w;
    twiddles(p.grid.n[a], w);
    CK_TRY(cudaMemcpy(p.tw[a], w.data(), w.size() * 8, cudaMemcpyHostToDevice));
    // y and z transform full lengths, x the half length
    stage_twiddles(a == 0 ? p.grid.n[0] / 2 : p.grid.n[a], w);
    if (w.size() > (size_t)p.grid.n[a]) return CK_ERR_ARG;
    CK_TRY(cudaMemcpy(p.stw[a], w.data(), w.size() * 8, cudaMemcpyHostToDevice));
  }
  {
    // w512^(l2 m1) with the 32 values of l2 adjacent: a warp of the K^ z
    // pass reads consecutive entries
    std::vector<float2> w(512);
    for (int m1 = 0; m1 < 16; ++m1)
      for (int l2 = 0; l2 < 32; ++l2) {
        const double a = 2.0 * M_PI * (double)(l2 * m1) / 512.0;
        w[(size_t)m1 * 32 + l2] = make_float2((float)cos(a), (float)-sin(a));
      }
    CK_TRY(cudaMemcpy(p.twm, w.data(), w.size() * 8, cudaMemcpyHostToDevice));
  }
  // dense [N_s]^(n-1) index -> rank of its sorted multiset
  std::vector<int> map((size_t)std::max<int64_t>(p.dense_total, 1), 0);
  for (int n = 2; n <= p.max_order; ++n) {
    const int k = n - 1;
    for (int64_t d = 0; d < p.dense_elems[n]; ++d) {
      int s[4];
      int64_t r = d;
      for (int i = k - 1; i >= 0; --i) {
        s[i] = (int)(r % p.ns);
        r /= p.ns;
      }
      std::sort(s, s + k);
      map[(size_t)(p.dense_base[n] + d)] = (int)host_multiset_rank(s, k, p.ns);
    }
  }
  CK_TRY(cudaMemcpy(p.dense_map, map.data(), map.size() * 4, cudaMemcpyHostToDevice));
  CK_TRY(cudaMemsetAsync(p.dstate, 0, sizeof(DevState), st));
  reset_state_kernel<<<1, 1, 0, st>>>(p.dstate, 0);
  reset_state_kernel<<<1, 1, 0, st>>>(p.dstate, 1);
  return cuda_status(cudaGetLastError());
}

// Grid one catalog (host or device positions) into counts[which].
// Grid field `which` (0 data, 1 randoms) from positions x, y, z and, when w
// is not NULL, per-point weights (all four in the same memory space).
// Page-locked host arrays that the device can address (mapped pinned
// memory) are read by the gridding kernel in place, over the host link;
// other host arrays stream through the staging slots.
// Only memory registered with the current device's context is read in place;
// page-locked memory of another device's context goes through staging.
const float* mapped_host(const float* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return nullptr;
  return a.type == cudaMemoryTypeHost && a.device == cur && a.devicePointer
             ? static_cast<const float*>(a.devicePointer)
             : nullptr;
}

ck_status grid_catalog(Plan& p, const float* x, const float* y, const float* z, int64_t n, int which,
                       cudaStream_t st, const float* w = nullptr) {
  CK_TRY(launch_clear_counts(p, which, st));  // before the box it reads is reset
  reset_state_kernel<<<1, 1, 0, st>>>(p.dstate, which);
  if (w) CK_TRY(cudaMemsetAsync(p.wacc, 0, (size_t)p.nc * 8, st));
  if (n > 0) {
    const bool dx = is_device_ptr(x), dy = is_device_ptr(y), dz = is_device_ptr(z);
    if (dx != dy || dx != dz || (w && is_device_ptr(w) != dx)) return CK_ERR_BAD_POINTER;
    auto grid = [&](const float* gx, const float* gy, const float* gz, const float* gw, int64_t cnt) {
      if (w) launch_grid_points_weighted(p, gx, gy, gz, gw, cnt, which, st);
      else launch_grid_points(p, gx, gy, gz, cnt, which, st);
    };
    const float* mx = dx ? nullptr : mapped_host(x);
    const float* my = mx ? mapped_host(y) : nullptr;
    const float* mz = my ? mapped_host(z) : nullptr;
    const float* mw = (mz && w) ? mapped_host(w) : nullptr;
    if (dx) {
      grid(x, y, z, w, n);
    } else if (mz && (!w || mw)) {
      grid(mx, my, mz, mw, n);  // pinned host arrays, read in place
    } else {
      // host positions (and weights): stream them through the staging slots
      int slot = 0;
      for (int64_t off = 0; off < n; off += p.staging_pts) {
        const int64_t cnt = std::min<int64_t>(p.staging_pts, n - off);
        float* sx = p.staging + (size_t)slot * 4 * p.staging_pts;
        float* sy = sx + p.staging_pts;
        float* sz = sy + p.staging_pts;
        float* sw = sz + p.staging_pts;
        CK_TRY(cudaMemcpyAsync(sx, x + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, st));
        CK_TRY(cudaMemcpyAsync(sy, y + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, st));
        CK_TRY(cudaMemcpyAsync(sz, z + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, st));
        if (w) CK_TRY(cudaMemcpyAsync(sw, w + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, st));
        grid(sx, sy, sz, sw, cnt);
        slot ^= 1;
      }
    }
  }
  if (w) launch_weights_to_cells(p, which, st);
  return cuda_status(cudaGetLastError());
}

// Convolve the current field with every shell kernel (Eqs. 9-10) and form
// the product sums of the orders in `mask` (Eq. 11) into `sums`: through the
// bank and the contraction kernels, or in one fused pass (fused plans, which
// always form every order up to max_order).
// W_0 is the transformed field itself, or w0 when given (cross-correlation).
// With a region set (ck_plan_set_region), W_0 = the field restricted to the
// region's planes: the whole field is transformed (the halo enters the
// convolution), then the planes outside the region are zeroed.
// support: 0 (a catalog: N = D - alpha R) or 1 (the randoms: Rt) lets the
// fused pass visit only the box of occupied cells, outside which W_0 = 0;
// -1 (fields given on the grid) visits every cell.
ck_status convolve_and_sum(Plan& p, int mask, double* sums, cudaStream_t st, const float* w0 = nullptr,
                           int support = -1) {
  if (!w0) w0 = p.field;
  if (support >= 0) launch_support_box(p, support, st);
  launch_fft_forward(p, p.field, p.spec, st, support >= 0 ? p.support + 6 : nullptr, true);
  if (p.region && w0 == p.field) {
    const size_t plane = (size_t)p.grid.n[0] * p.grid.n[1];
    if (p.region_z0 > 0) CK_TRY(cudaMemsetAsync(p.field, 0, plane * p.region_z0 * sizeof(float), st));
    if (p.region_z1 < p.grid.n[2])
      CK_TRY(cudaMemsetAsync(p.field + plane * p.region_z1, 0, plane * (p.grid.n[2] - p.region_z1) * sizeof(float),
                             st));
  }
  if (p.fused) return launch_convolve_contract(p, w0, sums, st, support >= 0 ? p.support : nullptr);
  // the bank on the planes the sums visit (W_0 vanishes outside them);
  // ck_get_bank and ck_product_map recompute whole fields
  launch_fft_inverse(p, p.spec, 0, p.ns, p.tmp, p.bank, p.field_stride, st, support >= 0 ? p.support : nullptr);
  return launch_contract(p, mask, w0, p.bank, p.field_stride, sums, st, support >= 0 ? p.support : nullptr);
}

int full_mask(const Plan& p) {
  int m = 0;
  for (int n = 2; n <= p.max_order; ++n) m |= 1 << n;
  return m;
}

ck_status read_status(Plan& p, cudaStream_t st, bool clear) {
  int h = 0;
  CK_TRY(cudaMemcpyAsync(&h, &p.dstate->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK_TRY(cudaStreamSynchronize(st));
  if (clear && h != 0) CK_TRY(cudaMemsetAsync(&p.dstate->status, 0, sizeof(int), st));
  return (ck_status)h;
}

ck_status copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st, bool* host_seen) {
  if (!dst) return CK_OK;
  if (is_device_ptr(dst)) {
    CK_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    *host_seen = true;
    CK_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  }
  return CK_OK;
}

// Copy the finalised outputs of the requested orders (and the dropped
// counts) to the caller's pointers; *host_seen is set for host destinations.
ck_status copy_results(Plan& p, int order_mask, const ck_outputs* out, cudaStream_t st, bool* host_seen) {
  if (!out) return CK_OK;
  for (int k = 2; k <= p.max_order; ++k) {
    if (!((order_mask >> k) & 1)) continue;
    const size_t bytes = (size_t)p.dense_elems[k] * 8;
    CK_TRY_S(copy_out(out->xi[k], p.dense + p.dense_base[k], bytes, st, host_seen));
    CK_TRY_S(copy_out(out->num[k], p.dense + p.dense_total + p.dense_base[k], bytes, st, host_seen));
    CK_TRY_S(copy_out(out->den[k], p.dense + 2 * p.dense_total + p.dense_base[k], bytes, st, host_seen));
  }
  CK_TRY_S(copy_out(out->dropped, p.dstate->dropped, 2 * sizeof(int64_t), st, host_seen));
  return CK_OK;
}

// Capture one catalog's compute sequence (gridding from p.dref through the
// finalised xi of order_mask) into an instantiated CUDA graph.
ck_status capture_compute(Plan& p, int order_mask) {
  if (p.gexec[order_mask]) return CK_OK;
  if (!p.fused) CK_TRY_S(contract_prepare(p, order_mask));  // its table uploads are synchronous
  if (!p.cap_stream) CK_TRY(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking));
  const bool prof = p.prof.on;
  p.prof.on = false;
  cudaStream_t cs = p.cap_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  ck_status s = CK_OK;
  if (e == cudaSuccess) {
    e = launch_clear_counts(p, 0, cs);
    reset_state_kernel<<<1, 1, 0, cs>>>(p.dstate, 0);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
      launch_grid_points_ref(p, 0, cs);
      launch_prepare_data(p, cs);
      s = convolve_and_sum(p, order_mask, p.sums, cs, nullptr, 0);
      if (s == CK_OK) launch_finalize(p, order_mask, cs);
    }
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
  }
  p.prof.on = prof;
  if (e == cudaSuccess && s == CK_OK) e = cudaGraphInstantiate(&p.gexec[order_mask], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (s != CK_OK) return s;
  return cuda_status(e);
}

}  // namespace

extern "C" {

int32_t ck_abi_version(void) { return CK_ABI_VERSION; }

const char* ck_status_string(ck_status s) {
  switch (s) {
    case CK_OK: return "ok";
    case CK_ERR_ARG: return "argument out of range";
    case CK_ERR_BAD_POINTER: return "bad pointer";
    case CK_ERR_OOM: return "out of device memory / workspace too small";
    case CK_ERR_EMPTY_SHELL: return "a shell contains no lattice offset";
    case CK_ERR_KERNEL_TOO_LARGE: return "shell kernel reaches half the box (offsets alias)";
    case CK_ERR_GUARD_BAND: return "occupied cells plus kernel reach exceed a non-periodic box";
    case CK_ERR_ZERO_DENOM: return "non-positive denominator (xi = NaN there)";
    case CK_ERR_TIMEOUT: return "a bounded device wait timed out";
    case CK_ERR_CUDA: return "CUDA runtime error";
    case CK_ERR_UNSUPPORTED: return "unsupported size or mode";
    case CK_ERR_NO_RANDOMS: return "ck_set_randoms has not been called";
    case CK_ERR_EMPTY_CATALOG: return "no point fell inside the grid";
  }
  return "unknown status";
}

ck_status ck_plan_workspace_size(const ck_grid* grid, const ck_shells* shells, int32_t max_order,
                                 int32_t precision, size_t* bytes) {
  if (!bytes) return CK_ERR_BAD_POINTER;
  Plan p;
  CK_TRY_S(validate_and_layout(grid, shells, max_order, precision, &p));
  *bytes = workspace_bytes(p);
  return CK_OK;
}

ck_status ck_plan_create(const ck_grid* grid, const ck_shells* shells, int32_t max_order, int32_t precision,
                         void* workspace, size_t workspace_bytes_in, void* stream, ck_plan** out) {
  if (!out) return CK_ERR_BAD_POINTER;
  *out = nullptr;
  Plan* p = new (std::nothrow) Plan();
  if (!p) return CK_ERR_OOM;
  ck_status s = validate_and_layout(grid, shells, max_order, precision, p);
  if (s != CK_OK) { delete p; return s; }
  const size_t need = workspace_bytes(*p);
  cudaStream_t st = S(stream);
  auto fail = [&](ck_status code) {
    if (p->owns_ws && p->ws) cudaFree(p->ws);
    delete p;
    return code;
  };
  // a caller workspace smaller than the plan needs is refused before any CUDA call
  if (workspace && workspace_bytes_in < need) return fail(CK_ERR_OOM);
  if (cudaGetDevice(&p->device) != cudaSuccess) return fail(CK_ERR_CUDA);
  if (cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    return fail(CK_ERR_CUDA);
  if (workspace) {
    if (((uintptr_t)workspace & 255u) != 0 || !is_device_ptr(workspace)) return fail(CK_ERR_BAD_POINTER);
    p->ws = workspace;
    p->ws_bytes = workspace_bytes_in;
  } else {
    cudaError_t e = cudaMalloc(&p->ws, need);
    if (e != cudaSuccess) { cudaGetLastError(); p->ws = nullptr; return fail(CK_ERR_OOM); }
    p->owns_ws = true;
    p->ws_bytes = need;
  }
  if ((s = carve(*p)) != CK_OK) return fail(s);
  if ((s = fft_init_attributes()) != CK_OK) return fail(s);
  if ((s = upload_tables(*p, st)) != CK_OK) return fail(s);
  if ((s = build_kernel_spectra(*p, st)) != CK_OK) return fail(s);
  *out = reinterpret_cast<ck_plan*>(p);
  return CK_OK;
}

ck_status ck_plan_destroy(ck_plan* plan) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan* p = reinterpret_cast<Plan*>(plan);
  cudaError_t e = cudaDeviceSynchronize();
  for (auto& r : p->prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (p->prof.pin) cudaFreeHost(p->prof.pin);
  for (auto& g : p->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->batch_stream) cudaStreamDestroy(p->batch_stream);
  if (p->batch_fork) cudaEventDestroy(p->batch_fork);
  if (p->batch_join) cudaEventDestroy(p->batch_join);
  if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
  if (p->aux_fork) cudaEventDestroy(p->aux_fork);
  if (p->aux_join) cudaEventDestroy(p->aux_join);
  if (p->owns_ws && p->ws) cudaFree(p->ws);
  delete p;
  return cuda_status(e);
}

ck_status ck_plan_get_info(const ck_plan* plan, ck_plan_info* info) {
  if (!plan || !info) return CK_ERR_BAD_POINTER;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  memset(info, 0, sizeof(*info));
  info->n_cells = p->nc;
  info->spec_pitch = p->px;
  info->n_shells = p->ns;
  info->max_order = p->max_order;
  for (int a = 0; a < 3; ++a) info->max_offset[a] = p->maxoff[a];
  for (int s = 0; s < p->ns; ++s) info->shell_size[s] = (int64_t)p->offsets[s].size() / 3;
  for (int n = 0; n <= CK_MAX_ORDER; ++n) info->n_multisets[n] = p->n_multisets[n];
  info->workspace_bytes = p->ws_bytes;
  info->bank_stride = p->field_stride;
  info->fused = p->fused ? 1 : 0;
  for (int a = 0; a < 3; ++a) info->fft_n[a] = p->grid.n[a];
  return CK_OK;
}

static ck_status set_randoms_impl(ck_plan* plan, const float* x, const float* y, const float* z, const float* w,
                                  int64_t n, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  if (n < 0) return CK_ERR_ARG;
  if (n > 0 && (!x || !y || !z)) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  cudaStream_t st = S(stream);
  p.have_randoms = p.have_randoms_diag = false;
  CK_TRY_S(grid_catalog(p, x, y, z, n, 1, st, w));
  launch_prepare_randoms(p, st);
  p.bank_holds = -1;
  CK_TRY_S(convolve_and_sum(p, full_mask(p), p.den_raw, st, nullptr, 1));
  p.bank_holds = 1;
  CK_TRY(cudaGetLastError());
  p.have_randoms = p.have_randoms_diag = true;
  return CK_OK;
}

ck_status ck_set_randoms(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n, void* stream) {
  return set_randoms_impl(plan, x, y, z, nullptr, n, stream);
}

ck_status ck_set_randoms_weighted(ck_plan* plan, const float* x, const float* y, const float* z, const float* w,
                                  int64_t n, void* stream) {
  if (n > 0 && !w) return CK_ERR_BAD_POINTER;
  return set_randoms_impl(plan, x, y, z, w, n, stream);
}

ck_status ck_set_randoms_factorised(ck_plan* plan, const ck_cosmology* cosmo, const ck_selection* sel,
                                    void* stream) {
  if (!plan || !cosmo || !sel) return CK_ERR_BAD_POINTER;
  CK_TRY_S(check_factorised(cosmo, sel));
  Plan& p = *reinterpret_cast<Plan*>(plan);
  cudaStream_t st = S(stream);
  p.have_randoms = p.have_randoms_diag = false;
  CK_TRY(launch_clear_counts(p, 1, st));
  reset_state_kernel<<<1, 1, 0, st>>>(p.dstate, 1);
  CK_TRY_S(launch_factorised_randoms(p, cosmo, sel, st));
  launch_prepare_randoms(p, st);
  p.bank_holds = -1;
  CK_TRY_S(convolve_and_sum(p, full_mask(p), p.den_raw, st, nullptr, 1));
  p.bank_holds = 1;
  CK_TRY(cudaGetLastError());
  p.have_randoms = p.have_randoms_diag = true;
  return CK_OK;
}

ck_status ck_set_randoms_diagonal(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n,
                                  void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  if (n < 0) return CK_ERR_ARG;
  if (n > 0 && (!x || !y || !z)) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  cudaStream_t st = S(stream);
  p.have_randoms = p.have_randoms_diag = false;
  CK_TRY_S(grid_catalog(p, x, y, z, n, 1, st));
  launch_prepare_randoms(p, st);
  p.bank_holds = -1;
  launch_fft_forward(p, p.field, p.spec, st, nullptr, true);
  bool full = false;
  CK_TRY_S(launch_diagonal_randoms(p, &full, st));
  p.bank_holds = 1;
  CK_TRY(cudaGetLastError());
  p.have_randoms = full;
  p.have_randoms_diag = true;
  return CK_OK;
}

static ck_status compute_impl(ck_plan* plan, const float* x, const float* y, const float* z, const float* w,
                              int64_t n, int32_t order_mask, const ck_outputs* out, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (n < 0) return CK_ERR_ARG;
  if (n > 0 && (!x || !y || !z)) return CK_ERR_BAD_POINTER;
  if (order_mask == 0 || (order_mask & ~full_mask(p)) != 0) return CK_ERR_ARG;
  if (!p.have_randoms) return CK_ERR_NO_RANDOMS;
  cudaStream_t st = S(stream);
  CK_TRY_S(grid_catalog(p, x, y, z, n, 0, st, w));
  launch_prepare_data(p, st);
  p.bank_holds = -1;
  CK_TRY_S(convolve_and_sum(p, order_mask, p.sums, st, nullptr, 0));
  p.bank_holds = 0;
  launch_finalize(p, order_mask, st);
  CK_TRY(cudaGetLastError());
  bool host_seen = false;
  CK_TRY_S(copy_results(p, order_mask, out, st, &host_seen));
  if (host_seen) return read_status(p, st, true);
  return CK_OK;
}

ck_status ck_compute(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n,
                     int32_t order_mask, const ck_outputs* out, void* stream) {
  return compute_impl(plan, x, y, z, nullptr, n, order_mask, out, stream);
}

ck_status ck_compute_weighted(ck_plan* plan, const float* x, const float* y, const float* z, const float* w,
                              int64_t n, int32_t order_mask, const ck_outputs* out, void* stream) {
  if (n > 0 && !w) return CK_ERR_BAD_POINTER;
  return compute_impl(plan, x, y, z, w, n, order_mask, out, stream);
}

// Fields on the grid (Secs. 2.7, 2.8): a0 (and b0) are loaded into the
// transformed field (continuous: Eq. 15's delta; cross: a copy of f1), f0
// into the W_0 buffer (the data count buffer) for a cross pair; then the
// plain sums of Eq. 16.  Host fields are first copied into the bank's first
// field (and b0 into the data count buffer), in box layout.  The randoms'
// grid, state and cached denominators are left as they are; the loaded
// fields' extent is kept as field 0's.
static ck_status fields_impl(ck_plan* plan, const float* a0, const float* b0, const float* f0, bool delta,
                             int32_t order_mask, const ck_outputs* out, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (!a0 || (!delta && !f0)) return CK_ERR_BAD_POINTER;
  if (order_mask == 0 || (order_mask & ~full_mask(p)) != 0) return CK_ERR_ARG;
  cudaStream_t st = S(stream);
  const size_t bytes = (size_t)p.box_n[0] * p.box_n[1] * p.box_n[2] * sizeof(float);
  // a host field lands in count buffer k (box layout) before it is loaded
  auto on_device = [&](const float* f, float* stage, const float** dev) -> ck_status {
    if (is_device_ptr(f)) {
      *dev = f;
      return CK_OK;
    }
    CK_TRY(cudaMemcpyAsync(stage, f, bytes, cudaMemcpyHostToDevice, st));
    *dev = stage;
    return CK_OK;
  };
  reset_state_kernel<<<1, 1, 0, st>>>(p.dstate, 0);
  // the data count buffer serves as staging and as W_0 below
  CK_TRY(cudaMemsetAsync(&p.dstate->counts_known[0], 0, sizeof(int), st));
  float* stage0 = p.bank;                                     // host a0 / f0 / f1
  float* stage1 = reinterpret_cast<float*>(p.counts[0]);      // host b0
  const bool padded = p.grid.n[0] != p.box_n[0] || p.grid.n[1] != p.box_n[1] || p.grid.n[2] != p.box_n[2];
  if (padded) CK_TRY(cudaMemsetAsync(p.field, 0, (size_t)p.nc * 4, st));
  float* w0 = nullptr;
  if (!delta) {  // W_0 = f0 in the data count buffer, stored layout
    const float* d0 = nullptr;
    CK_TRY_S(on_device(f0, stage0, &d0));
    w0 = reinterpret_cast<float*>(p.counts[0]);
    if (padded) CK_TRY(cudaMemsetAsync(w0, 0, (size_t)p.nc * 4, st));
    launch_field_load(p, d0, nullptr, false, w0, 0, st);
  }
  const float* da = nullptr;
  const float* db = nullptr;
  CK_TRY_S(on_device(a0, stage0, &da));
  if (b0) CK_TRY_S(on_device(b0, stage1, &db));
  launch_field_load(p, da, db, delta, p.field, 0, st);
  // the loaded field may be nonzero anywhere: the next preparation rewrites every plane
  CK_TRY(cudaMemsetAsync(&p.dstate->field_known, 0, sizeof(int), st));
  launch_field_check(p, st);
  p.bank_holds = -1;
  CK_TRY_S(convolve_and_sum(p, order_mask, p.sums, st, w0));
  p.bank_holds = 2;  // a field's convolutions (not a catalog's)
  launch_finalize(p, order_mask, st, true);
  CK_TRY(cudaGetLastError());
  bool host_seen = false;
  CK_TRY_S(copy_results(p, order_mask, out, st, &host_seen));
  if (host_seen) return read_status(p, st, true);
  return CK_OK;
}

ck_status ck_compute_continuous(ck_plan* plan, const float* d, const float* r, int32_t order_mask,
                                const ck_outputs* out, void* stream) {
  return fields_impl(plan, d, r, nullptr, true, order_mask, out, stream);
}

ck_status ck_compute_cross(ck_plan* plan, const float* f0, const float* f1, int32_t order_mask,
                           const ck_outputs* out, void* stream) {
  if (!plan || !f0 || !f1) return CK_ERR_BAD_POINTER;
  return fields_impl(plan, f1, nullptr, f0, false, order_mask, out, stream);
}

ck_status ck_product_map(ck_plan* plan, int32_t shell, float* map, void* stream) {
  if (!plan || !map) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (shell < 0 || shell >= p.ns) return CK_ERR_ARG;
  if (!p.have_randoms_diag) return CK_ERR_NO_RANDOMS;
  if (p.bank_holds != 0) return CK_ERR_ARG;  // needs a catalog's ck_compute just before
  cudaStream_t st = S(stream);
  // recompute W_s from the resident spectrum: fused plans keep no bank, and
  // a catalog's bank holds only the planes its sums visited
  float* ws = p.fused ? p.bank : p.bank + (size_t)shell * p.field_stride;
  launch_fft_inverse(p, p.spec, shell, 1, p.tmp, ws, p.field_stride, st);
  const bool dev = is_device_ptr(map);
  const size_t bytes = (size_t)p.box_n[0] * p.box_n[1] * p.box_n[2] * sizeof(float);
  float* dst = dev ? map : reinterpret_cast<float*>(p.counts[0]);  // host: through the data count buffer
  if (!dev) CK_TRY(cudaMemsetAsync(&p.dstate->counts_known[0], 0, sizeof(int), st));
  launch_product_map(p, p.field, ws, shell, dst, st);
  CK_TRY(cudaGetLastError());
  if (!dev) {
    CK_TRY(cudaMemcpyAsync(map, dst, bytes, cudaMemcpyDeviceToHost, st));
    CK_TRY(cudaStreamSynchronize(st));
    return read_status(p, st, true);
  }
  return CK_OK;
}

ck_status ck_compute_diagonal(ck_plan* plan, const float* x, const float* y, const float* z, int64_t n,
                              int32_t order_mask, const ck_outputs* out, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (n < 0) return CK_ERR_ARG;
  if (n > 0 && (!x || !y || !z)) return CK_ERR_BAD_POINTER;
  if (order_mask == 0 || (order_mask & ~full_mask(p)) != 0) return CK_ERR_ARG;
  if (!p.have_randoms_diag) return CK_ERR_NO_RANDOMS;
  cudaStream_t st = S(stream);
  CK_TRY_S(grid_catalog(p, x, y, z, n, 0, st));
  launch_prepare_data(p, st);
  p.bank_holds = -1;
  launch_fft_forward(p, p.field, p.spec, st, nullptr, true);
  CK_TRY_S(launch_diagonal(p, order_mask, st));
  p.bank_holds = 0;
  CK_TRY(cudaGetLastError());
  bool host_seen = false;
  if (out) {
    for (int k = 2; k <= p.max_order; ++k) {
      if (!((order_mask >> k) & 1)) continue;
      const size_t bytes = (size_t)p.ns * 8;
      CK_TRY_S(copy_out(out->xi[k], p.dense + p.dense_base[k], bytes, st, &host_seen));
      CK_TRY_S(copy_out(out->num[k], p.dense + p.dense_total + p.dense_base[k], bytes, st, &host_seen));
      CK_TRY_S(copy_out(out->den[k], p.dense + 2 * p.dense_total + p.dense_base[k], bytes, st, &host_seen));
    }
    CK_TRY_S(copy_out(out->dropped, p.dstate->dropped, 2 * sizeof(int64_t), st, &host_seen));
  }
  if (host_seen) return read_status(p, st, true);
  return CK_OK;
}

ck_status ck_batch_compute(ck_plan* const* plans, int32_t n_plans, const ck_catalog* cats, int32_t n_cats,
                           int32_t order_mask, const ck_outputs* out, void* stream) {
  if (!plans || !cats || n_plans < 1 || n_cats < 0) return n_plans < 1 || n_cats < 0 ? CK_ERR_ARG : CK_ERR_BAD_POINTER;
  if (n_cats == 0) return CK_OK;
  for (int32_t j = 0; j < n_plans; ++j)
    if (!plans[j]) return CK_ERR_BAD_POINTER;
  for (int32_t i = 0; i < n_cats; ++i) {
    const ck_catalog& c = cats[i];
    if (c.plan < 0 || c.plan >= n_plans || c.n < 0) return CK_ERR_ARG;
    Plan& p = *reinterpret_cast<Plan*>(plans[c.plan]);
    if (order_mask == 0 || (order_mask & ~full_mask(p)) != 0) return CK_ERR_ARG;
    if (!p.have_randoms) return CK_ERR_NO_RANDOMS;
    if (c.n > 0 && (!c.x || !c.y || !c.z)) return CK_ERR_BAD_POINTER;
    if (c.n > 0 && (!is_device_ptr(c.x) || !is_device_ptr(c.y) || !is_device_ptr(c.z))) return CK_ERR_BAD_POINTER;
  }
  cudaStream_t st = S(stream);
  std::vector<char> used((size_t)n_plans, 0);
  int n_used = 0;
  for (int32_t i = 0; i < n_cats; ++i)
    if (!used[(size_t)cats[i].plan]) {
      used[(size_t)cats[i].plan] = 1;
      ++n_used;
    }
  for (int32_t j = 0; j < n_plans; ++j)
    if (used[(size_t)j]) CK_TRY_S(capture_compute(*reinterpret_cast<Plan*>(plans[j]), order_mask));
  // Several plans (grid classes): each plan's catalogs in order on the
  // plan's own stream, so that the classes run concurrently (they share no
  // buffers), joined back to the caller's stream at the end.
  const bool fork = n_used > 1;
  if (fork)
    for (int32_t j = 0; j < n_plans; ++j) {
      if (!used[(size_t)j]) continue;
      Plan& p = *reinterpret_cast<Plan*>(plans[j]);
      if (!p.batch_stream) CK_TRY(cudaStreamCreateWithFlags(&p.batch_stream, cudaStreamNonBlocking));
      if (!p.batch_fork) CK_TRY(cudaEventCreateWithFlags(&p.batch_fork, cudaEventDisableTiming));
      if (!p.batch_join) CK_TRY(cudaEventCreateWithFlags(&p.batch_join, cudaEventDisableTiming));
      CK_TRY(cudaEventRecord(p.batch_fork, st));
      CK_TRY(cudaStreamWaitEvent(p.batch_stream, p.batch_fork, 0));
    }
  bool host_seen = false;
  ck_status s = CK_OK;
  for (int32_t i = 0; i < n_cats && s == CK_OK; ++i) {
    Plan& p = *reinterpret_cast<Plan*>(plans[cats[i].plan]);
    cudaStream_t ps = fork ? p.batch_stream : st;
    launch_set_catalog_ref(p, cats[i].x, cats[i].y, cats[i].z, cats[i].n, ps);
    s = cuda_status(cudaGraphLaunch(p.gexec[order_mask], ps));
    p.bank_holds = 0;
    if (s == CK_OK) s = copy_results(p, order_mask, out ? out + i : nullptr, ps, &host_seen);
  }
  // the plan streams join the caller's stream even after an error, so that
  // later work on it is ordered after everything launched here
  if (fork)
    for (int32_t j = 0; j < n_plans; ++j) {
      if (!used[(size_t)j]) continue;
      Plan& p = *reinterpret_cast<Plan*>(plans[j]);
      const ck_status r = cuda_status(cudaEventRecord(p.batch_join, p.batch_stream));
      const ck_status w = r == CK_OK ? cuda_status(cudaStreamWaitEvent(st, p.batch_join, 0)) : r;
      if (s == CK_OK) s = w;
    }
  CK_TRY_S(s);
  CK_TRY(cudaGetLastError());
  if (host_seen) {
    ck_status first = CK_OK;
    for (int32_t j = 0; j < n_plans; ++j) {
      const ck_status s = read_status(*reinterpret_cast<Plan*>(plans[j]), st, true);
      if (first == CK_OK) first = s;
    }
    return first;
  }
  return CK_OK;
}

// Autotuning: each candidate of a choice runs once to warm up and five
// times between events on the plan's own buffers; the candidate with the
// fastest run is kept.
ck_status ck_plan_autotune(ck_plan* plan, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (p.bank_holds < 0) return CK_ERR_NO_RANDOMS;  // no resident field to time on
  cudaStream_t st = S(stream);
  const bool prof = p.prof.on;
  p.prof.on = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck_status s = cuda_status(cudaEventCreate(&e0));
  if (s == CK_OK) s = cuda_status(cudaEventCreate(&e1));
  // once untimed, then the fastest of five timed runs (robust to other work on the GPU)
  auto timed = [&](auto&& fn, float* ms) -> ck_status {
    fn();
    *ms = 1e30f;
    for (int r = 0; r < 5; ++r) {
      CK_TRY(cudaEventRecord(e0, st));
      fn();
      CK_TRY(cudaEventRecord(e1, st));
      CK_TRY(cudaEventSynchronize(e1));
      float t = 0.0f;
      CK_TRY(cudaEventElapsedTime(&t, e0, e1));
      *ms = std::min(*ms, t);
    }
    return cuda_status(cudaGetLastError());
  };
  const int ny = p.grid.n[1], nz = p.grid.n[2];
  // a catalog's field (after ck_set_randoms or a compute): the passes visit
  // its support box, as in the step itself (the pruned forward transform
  // gives the same spectrum); a loaded field: every plane and row
  const int* box = (p.bank_holds == 0 || p.bank_holds == 1) ? p.support : nullptr;
  // the z step (the direct filter, where the plan has one, or the K^ z
  // pass) with the forward transform each needs, and the tile widths of
  // the 512-point register passes under each: the single-field strided
  // passes, then the K^ z pass with the multi-shell inverse y pass; the
  // route with the faster forward + inverse z and y passes is kept
  if (s == CK_OK) {
    const Tuning orig = p.tune;
    Tuning win = p.tune;
    float best = 1e30f;
    for (int zd = 0; zd <= 1 && s == CK_OK; ++zd) {
      if (zd == 1 && p.kz_dz == 0) break;
      p.tune.z_direct = zd;
      float fbest = 1e30f, ibest = 1e30f;
      int fc = orig.fwd_cols, pz = orig.zreg_cols, py = orig.yinv_cols;
      for (int c : {8, 16}) {
        if (ny != 512 && nz != 512 && c != orig.fwd_cols) continue;
        p.tune.fwd_cols = c;
        float ms = 0.0f;
        if ((s = timed([&] { launch_fft_forward(p, p.field, p.spec, st, box ? box + 6 : nullptr, true); }, &ms)) !=
            CK_OK)
          break;
        if (ms < fbest) { fbest = ms; fc = c; }
      }
      if (s != CK_OK) break;
      p.tune.fwd_cols = fc;  // the spectrum is in this route's form (every width gives the same)
      for (int cz : {8, 16})
        for (int cy : {8, 16}) {
          if (s != CK_OK) break;
          if ((zd == 1 || nz != 512) && cz != orig.zreg_cols) continue;
          if (ny != 512 && cy != orig.yinv_cols) continue;
          p.tune.zreg_cols = cz;
          p.tune.yinv_cols = cy;
          float ms = 0.0f;
          if ((s = timed([&] { launch_inverse_zy(p, p.spec, 0, p.ns, p.tmp, st, box); }, &ms)) != CK_OK) break;
          if (ms < ibest) { ibest = ms; pz = cz; py = cy; }
        }
      if (s == CK_OK && fbest + ibest < best) {
        best = fbest + ibest;
        win.z_direct = zd;
        win.fwd_cols = fc;
        win.zreg_cols = pz;
        win.yinv_cols = py;
      }
    }
    p.tune.z_direct = win.z_direct;
    p.tune.fwd_cols = win.fwd_cols;
    p.tune.zreg_cols = win.zreg_cols;
    p.tune.yinv_cols = win.yinv_cols;
  }
  // the tensor-core contraction's splits, on the randoms' bank
  const bool tensor = p.precision == CK_PREC_SPLIT_TF32 || p.precision == CK_PREC_SPLIT_BF16 ||
                      p.precision == CK_PREC_SPLIT_FP16;
  if (s == CK_OK && tensor && !p.fused) {
    const int mask = full_mask(p);
    // the widest stacked tile, then the CTAs per SM
    auto pick_best = [&](int* knob, std::initializer_list<int> cands) {
      float best = 1e30f;
      int pick = *knob;
      for (int k : cands) {
        *knob = k;
        for (bool& r : p.cplan_ready) r = false;
        float ms = 0.0f;
        const ck_status c =
            timed([&] { launch_contract(p, mask, p.field, p.bank, p.field_stride, p.sums, st, box); }, &ms);
        if (c == CK_ERR_OOM) continue;  // more splits than the partials hold
        if ((s = c) != CK_OK) break;
        if (ms < best) { best = ms; pick = k; }
      }
      *knob = pick;
    };
    pick_best(&p.tune.tc_stack_cols, {0, 32, 64});
    if (s == CK_OK) pick_best(&p.tune.tc_ctas_per_sm, {1, 2, 3});
    if (s == CK_OK) pick_best(&p.tune.tc_thin_overlap, {0, 1});
    for (bool& r : p.cplan_ready) r = false;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  p.prof.on = prof;
  // captured graphs hold the previous choices; a region's field no longer
  // gives the randoms' whole spectrum
  for (auto& g : p.gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (p.region) p.bank_holds = -1;
  if (s == CK_OK) {
    p.tune.tuned = true;
    s = read_status(p, st, false);
  }
  return s;
}

ck_status ck_plan_set_tuning(ck_plan* plan, const int32_t* in) {
  if (!plan || !in) return CK_ERR_BAD_POINTER;
  for (int i = 0; i < 3; ++i)
    if (in[i] != 8 && in[i] != 16) return CK_ERR_ARG;
  if (in[3] < 1 || in[3] > 3 || in[4] < 0 || in[4] > 128 || (in[5] != 0 && in[5] != 1) || (in[6] != 0 && in[6] != 1))
    return CK_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  p.tune.fwd_cols = in[0];
  p.tune.zreg_cols = in[1];
  p.tune.yinv_cols = in[2];
  p.tune.tc_ctas_per_sm = in[3];
  p.tune.tc_stack_cols = in[4];
  p.tune.tc_thin_overlap = in[5];
  p.tune.z_direct = in[6];
  for (bool& r : p.cplan_ready) r = false;
  for (auto& g : p.gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return CK_OK;
}

ck_status ck_plan_get_tuning(const ck_plan* plan, int32_t* out) {
  if (!plan || !out) return CK_ERR_BAD_POINTER;
  const Plan& p = *reinterpret_cast<const Plan*>(plan);
  out[0] = p.tune.fwd_cols;
  out[1] = p.tune.zreg_cols;
  out[2] = p.tune.yinv_cols;
  out[3] = p.tune.tc_ctas_per_sm;
  out[4] = p.tune.tc_stack_cols;
  out[5] = p.tune.tc_thin_overlap;
  out[6] = p.tune.z_direct && p.kz_dz > 0 ? 1 : 0;
  out[7] = p.tune.tuned ? 1 : 0;
  return CK_OK;
}

ck_status ck_plan_set_region(ck_plan* plan, int32_t z_begin, int32_t z_end, double alpha) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (z_begin < 0 || z_end <= z_begin || z_end > p.box_n[2]) return CK_ERR_ARG;
  if (!(alpha >= 0.0) || !isfinite(alpha)) return CK_ERR_ARG;
  p.region = !(z_begin == 0 && z_end == p.box_n[2] && alpha == 0.0);
  p.region_z0 = z_begin;
  p.region_z1 = z_end;
  p.region_alpha = alpha;
  // the captured compute graphs hold the previous setting
  for (auto& g : p.gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  // den_raw of the randoms set so far summed over other planes
  p.have_randoms = false;
  p.bank_holds = -1;
  p.have_randoms_diag = false;
  return CK_OK;
}

ck_status ck_plan_status(ck_plan* plan, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  return read_status(*reinterpret_cast<Plan*>(plan), S(stream), true);
}

const char* ck_stage_name(int32_t stage) {
  return (stage >= 0 && stage < CK_STAGES) ? kStageNames[stage] : nullptr;
}

ck_status ck_profile_enable(ck_plan* plan, int32_t enable) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  Profiler& f = p.prof;
  if (enable && f.recs.empty()) {
    f.recs.resize(kProfPool);
    for (auto& r : f.recs) {
      CK_TRY(cudaEventCreate(&r.a));
      CK_TRY(cudaEventCreate(&r.b));
    }
    CK_TRY(cudaHostAlloc(reinterpret_cast<void**>(&f.pin), kProfPool * 6 * sizeof(int), cudaHostAllocDefault));
  }
  if (f.used) CK_TRY(cudaDeviceSynchronize());
  f.used = 0;
  f.dropped = 0;
  for (int i = 0; i < CK_STAGES; ++i) {
    f.ms[i] = 0.0;
    f.launches[i] = 0;
    f.bytes[i] = 0.0;
  }
  f.on = enable != 0;
  return CK_OK;
}

ck_status ck_profile_read(ck_plan* plan, ck_stage_times* out) {
  if (!plan || !out) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  prof_collect(p);
  for (int i = 0; i < CK_STAGES; ++i) {
    out->ms[i] = p.prof.ms[i];
    out->launches[i] = p.prof.launches[i];
    out->bytes[i] = p.prof.bytes[i];
  }
  return CK_OK;
}

ck_status ck_get_grids(ck_plan* plan, uint32_t* d_counts, uint32_t* r_counts, void* stream) {
  if (!plan) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  cudaStream_t st = S(stream);
  bool host = false;
  CK_TRY_S(copy_out(d_counts, p.counts[0], (size_t)p.nc * 4, st, &host));
  CK_TRY_S(copy_out(r_counts, p.counts[1], (size_t)p.nc * 4, st, &host));
  if (host) CK_TRY(cudaStreamSynchronize(st));
  return CK_OK;
}

ck_status ck_get_field(ck_plan* plan, int32_t which, float* out, void* stream) {
  if (!plan || !out) return CK_ERR_BAD_POINTER;
  if (which != 0 && which != 1) return CK_ERR_ARG;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  // the field buffer holds the last stage's input (a loaded field counts as data)
  if (which != (p.bank_holds == 2 ? 0 : p.bank_holds)) return CK_ERR_ARG;
  cudaStream_t st = S(stream);
  bool host = false;
  CK_TRY_S(copy_out(out, p.field, (size_t)p.nc * 4, st, &host));
  if (host) CK_TRY(cudaStreamSynchronize(st));
  return CK_OK;
}

ck_status ck_get_bank(ck_plan* plan, int32_t shell, float* out, void* stream) {
  if (!plan || !out) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (shell < 0 || shell >= p.ns || p.bank_holds < 0) return CK_ERR_ARG;
  cudaStream_t st = S(stream);
  bool host = false;
  // recompute W_s from the resident spectrum: fused plans keep no bank, and
  // a catalog's bank holds only the planes its sums visited
  float* src = p.fused ? p.bank : p.bank + (size_t)shell * p.field_stride;
  launch_fft_inverse(p, p.spec, shell, 1, p.tmp, src, p.field_stride, st);
  CK_TRY(cudaGetLastError());
  CK_TRY_S(copy_out(out, src, (size_t)p.nc * 4, st, &host));
  if (host) CK_TRY(cudaStreamSynchronize(st));
  return CK_OK;
}

ck_status ck_get_kernel_spectrum(ck_plan* plan, int32_t shell, float* out, void* stream) {
  if (!plan || !out) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (shell < 0 || shell >= p.ns) return CK_ERR_ARG;
  cudaStream_t st = S(stream);
  const bool dev = is_device_ptr(out);
  // strip the row padding: pitch px -> n[0]/2 + 1
  CK_TRY(cudaMemcpy2DAsync(out, (size_t)p.oct[0] * 4, p.khat + (size_t)shell * p.khat_stride, (size_t)p.px * 4,
                           (size_t)p.oct[0] * 4, (size_t)p.oct[1] * p.oct[2],
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!dev) CK_TRY(cudaStreamSynchronize(st));
  return CK_OK;
}

ck_status ck_fft_r2c(ck_plan* plan, const float* in, void* out_spec, void* stream) {
  if (!plan || !in || !out_spec) return CK_ERR_BAD_POINTER;
  if (!is_device_ptr(in) || !is_device_ptr(out_spec)) return CK_ERR_BAD_POINTER;
  if (((uintptr_t)out_spec & 15u) != 0 || ((uintptr_t)in & 15u) != 0) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  launch_fft_forward(p, in, static_cast<float2*>(out_spec), S(stream));
  return cuda_status(cudaGetLastError());
}

ck_status ck_fft_c2r(ck_plan* plan, const void* in_spec, float* out, void* stream) {
  if (!plan || !in_spec || !out) return CK_ERR_BAD_POINTER;
  if (!is_device_ptr(in_spec) || !is_device_ptr(out)) return CK_ERR_BAD_POINTER;
  if (((uintptr_t)in_spec & 15u) != 0 || ((uintptr_t)out & 15u) != 0) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  launch_fft_inverse(p, static_cast<const float2*>(in_spec), -1, 1, p.tmp, out, 0, S(stream));
  return cuda_status(cudaGetLastError());
}

ck_status ck_contract(ck_plan* plan, const float* w0, const float* bank, int64_t bank_stride, int32_t order_mask,
                      double* const* sums, void* stream) {
  if (!plan || !w0 || !bank || !sums) return CK_ERR_BAD_POINTER;
  Plan& p = *reinterpret_cast<Plan*>(plan);
  if (order_mask == 0 || (order_mask & ~full_mask(p)) != 0) return CK_ERR_ARG;
  if (bank_stride < p.nc || (bank_stride % 4) != 0) return CK_ERR_ARG;
  if (((uintptr_t)w0 & 15u) != 0 || ((uintptr_t)bank & 15u) != 0) return CK_ERR_BAD_POINTER;
  if (!is_device_ptr(w0) || !is_device_ptr(bank)) return CK_ERR_BAD_POINTER;
  cudaStream_t st = S(stream);
  CK_TRY_S(launch_contract(p, order_mask, w0, bank, bank_stride, p.sums, st));
  bool host = false;
  for (int k = 2; k <= p.max_order; ++k) {
    if (!((order_mask >> k) & 1) || !sums[k]) continue;
    CK_TRY_S(copy_out(sums[k], p.sums + p.multiset_base[k], (size_t)p.n_multisets[k] * 8, st, &host));
  }
  if (host) CK_TRY(cudaStreamSynchronize(st));
  return CK_OK;
}

}  // extern "C"
