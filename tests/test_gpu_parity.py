"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: gridding is integer work and must match bit for bit.  Floating
point: the normwise error |x_gpu - x_ref| / sum_r |terms| of every product
sum (num and den) must be <= 1e-5 (FP32 FFTs and FP32 products with FP64
cross-block sums); convolution banks are compared relative to max |W|.
"""
import itertools
import math

import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, lattice_catalog, neyman_scott_box, uniform_box, workload
from tests.gpu_util import cuda_torch, dev, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


@pytest.fixture(scope="module")
def p32():
    return workload("periodic32")


@pytest.fixture(scope="module")
def ref32(p32):
    return O.correlate(p32["grid"], p32["shells"], p32["width"], p32["data"], p32["randoms"],
                       orders=(2, 3, 4, 5), engine="direct")


def _run(torch, w, orders, max_order=None, precision="fp32"):
    plan = plan_for(w, max_order=max_order or max(orders), precision=precision)
    plan.set_randoms(*dev_cat(torch, w["randoms"]))
    res = plan.compute(*dev_cat(torch, w["data"]), orders=orders, out="host")
    return plan, res


def _check_sums(res, ref, ns, orders, tol=TOL):
    for n in orders:
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
            e = normwise(got, want, scale)
            assert e <= tol, f"order {n} {key}: normwise error {e:.3e}"


# ---------------------------------------------------------------------------
# mapping

def test_gridding_periodic32_exact(torch, p32, ref32):
    plan, res = _run(torch, p32, (2,))
    d, r = plan.grids()
    assert np.array_equal(d.cpu().numpy().astype(np.uint32), ref32["D"])
    assert np.array_equal(r.cpu().numpy().astype(np.uint32), ref32["R"])
    assert res["dropped"].tolist() == [0, 0]


def test_gridding_edges_exact(torch):
    """Points on cell edges, just below them, at x = L and at negative
    coordinates (periodic), and outside a non-periodic box."""
    rng = np.random.default_rng(3)
    for periodic in (True, False):
        g = GridSpec((12, 10, 8), (-7.5, 3.25, 100.0), 2.5, periodic)
        cells = np.stack([rng.integers(0, g.n[a], 400) for a in range(3)], 1)
        edge = lattice_catalog(g, cells, where="edge")
        below = Catalog(np.nextafter(edge.x, np.float32(-np.inf)), edge.y, np.nextafter(edge.z, np.float32(np.inf)))
        L = np.array(g.length)
        far = Catalog(np.float32(g.origin[0]) + rng.uniform(-2 * L[0], 3 * L[0], 300).astype(np.float32),
                      np.float32(g.origin[1]) + rng.uniform(0, L[1], 300).astype(np.float32),
                      np.float32(g.origin[2]) + rng.uniform(-L[2], L[2], 300).astype(np.float32))
        ends = Catalog(np.float32(np.array([g.origin[0] + L[0]] * 3)), np.float32(np.array([g.origin[1]] * 3)),
                       np.float32(np.array([g.origin[2] + L[2] - 1e-4] * 3)))
        cat = Catalog.concat([edge, below, far, ends, lattice_catalog(g, cells)])
        want, wdrop = O.grid_counts(cat.x, cat.y, cat.z, g)
        w = dict(grid=g, shells=(2.6,), width=1.0, data=cat, randoms=cat)
        plan = plan_for(w, max_order=2)
        plan.set_randoms(*dev_cat(torch, cat))
        dropped = torch.zeros(2, dtype=torch.int64)
        outs = {k: {2: torch.empty(1, dtype=torch.float64)} for k in ("xi", "num", "den")}
        outs["dropped"] = dropped
        from paper_2108_00015_gb300 import CkError
        try:
            plan.compute(*dev_cat(torch, cat), orders=(2,), out="host", outputs=outs)
        except CkError as e:  # the points fill the box: a non-periodic grid reports its guard band
            assert not periodic and e.code == 6
        d, r = plan.grids()
        assert np.array_equal(d.cpu().numpy().astype(np.uint32), want)
        assert np.array_equal(r.cpu().numpy().astype(np.uint32), want)
        assert dropped.tolist() == [wdrop, wdrop]
        plan.close()


def test_gridding_survey_sample_exact(torch):
    w = workload("survey512", scale=0.05)
    g = w["grid"]
    plan = plan_for(w, max_order=2)
    plan.set_randoms(*dev_cat(torch, w["randoms"]))
    plan.compute(*dev_cat(torch, w["data"]), orders=(2,), out="host")
    d, r = plan.grids()
    D, _ = O.grid_counts(w["data"].x, w["data"].y, w["data"].z, g)
    R, _ = O.grid_counts(w["randoms"].x, w["randoms"].y, w["randoms"].z, g)
    assert np.array_equal(d.cpu().numpy().astype(np.uint32), D)
    assert np.array_equal(r.cpu().numpy().astype(np.uint32), R)
    plan.close()


# ---------------------------------------------------------------------------
# FFT

@pytest.mark.parametrize("shape", [(32, 32, 32), (18, 20, 24), (40, 30, 16), (80, 48, 64), (10, 6, 12),
                                   (128, 96, 160), (16, 384, 4), (240, 12, 288), (512, 4, 320),
                                   (160, 160, 160), (256, 256, 256), (16, 512, 64), (512, 16, 32),
                                   (512, 512, 16), (6, 10, 512), (16, 32, 512), (4, 4, 512)])
def test_fft_vs_numpy(torch, shape):
    nz, ny, nx = shape
    g = GridSpec((nx, ny, nz), (0.0, 0.0, 0.0), 1.0, True)
    w = dict(grid=g, shells=(1.0,), width=1.0)
    plan = plan_for(w, max_order=2)
    rng = np.random.default_rng(nx * 7 + ny)
    x = rng.normal(size=shape).astype(np.float32)
    spec = plan.fft_r2c(dev(torch, x)).cpu().numpy()[:, :, : nx // 2 + 1]
    want = np.fft.rfftn(x.astype(np.float64))
    e = np.abs(spec - want).max() / np.abs(want).max()
    assert e < 2e-6, f"forward error {e:.2e}"
    # inverse (unnormalised) of a Hermitian spectrum
    Xh = np.zeros((nz, ny, plan.spec_pitch), np.complex64)
    Xh[:, :, : nx // 2 + 1] = want.astype(np.complex64)
    back = plan.fft_c2r(dev(torch, Xh)).cpu().numpy()
    e2 = np.abs(back / x.size - x).max() / np.abs(x).max()
    assert e2 < 2e-6, f"inverse error {e2:.2e}"
    plan.close()


# ---------------------------------------------------------------------------
# kernels and convolution

def test_kernel_spectrum(torch, p32):
    g = p32["grid"]
    plan = plan_for(p32)
    for s, rad in enumerate(p32["shells"]):
        offs = O.shell_offsets(rad, p32["width"], g.cell)
        assert plan.shell_size[s] == offs.shape[0]
        want = O.kernel_spectrum_octant(offs, g.n)
        got = plan.kernel_spectrum(s).cpu().numpy()
        assert np.abs(got - want).max() <= 1e-6 * offs.shape[0] / g.n_cells + 1e-9
    plan.close()


def test_bank_periodic32(torch, p32, ref32):
    plan, _ = _run(torch, p32, (2,))
    N = plan.field(0).cpu().numpy()
    assert np.abs(N - ref32["N"]).max() <= 1e-6 * np.abs(ref32["N"]).max()
    for s in range(len(p32["shells"])):
        got = plan.bank(s).cpu().numpy()
        want = ref32["W"][s]
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), f"shell {s}"
    plan.close()


# ---------------------------------------------------------------------------
# summation and xi

def test_xi_periodic32_all_orders(torch, p32, ref32):
    plan, res = _run(torch, p32, (2, 3, 4, 5))
    _check_sums(res, ref32, len(p32["shells"]), (2, 3, 4, 5))
    for n in (2, 3, 4, 5):
        xi = res["xi"][n].numpy()
        want = ref32[f"xi{n}"]
        den = O.dense_tensor(ref32[f"den{n}"], 4, n - 1)
        bound = TOL * (O.dense_tensor(ref32[f"abs_num{n}"], 4, n - 1)
                       + np.abs(want) * O.dense_tensor(ref32[f"abs_den{n}"], 4, n - 1)) / den
        assert np.all(np.abs(xi - want) <= 2 * bound + 1e-300), f"xi order {n}"
    plan.close()


def test_xi_fp64_contraction(torch, p32, ref32):
    plan, res = _run(torch, p32, (2, 3, 4, 5), precision="fp64")
    _check_sums(res, ref32, len(p32["shells"]), (2, 3, 4, 5))
    plan.close()


# Gates of the split tensor-core forms: hi + lo operands carry 21-22
# significant bits in TF32 and FP16 (scaled per factor) and 16 in BF16, whose
# dropped lo*lo term and the rounding of lo leave about 2^-16 per product.
SPLIT_TOL = {"split_tf32": TOL, "split_fp16": TOL, "split_bf16": 5e-5}


@pytest.mark.parametrize("precision", ["split_tf32", "split_bf16", "split_fp16"])
def test_xi_split_all_orders(torch, p32, ref32, precision):
    """Mixed forms with orders up to 5: the bank is kept and every order runs
    through the tensor-core blocked product (kind::tf32, or kind::f16 with
    BF16 or FP16 hi/lo operands)."""
    plan, res = _run(torch, p32, (2, 3, 4, 5), precision=precision)
    assert not plan.fused
    _check_sums(res, ref32, len(p32["shells"]), (2, 3, 4, 5), tol=SPLIT_TOL[precision])
    plan.close()


@pytest.mark.parametrize("precision", ["split_tf32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("ns,dims", [(16, (24, 20, 18)), (20, (24, 20, 18)), (8, (30, 18, 10)), (12, (30, 18, 10))])
def test_tc_blocked_contraction(torch, ns, dims, precision):
    """The tensor-core blocked product over a caller's bank, orders 2..5,
    against the oracle's product sums of the same float32 fields, in each
    split form.  The shell counts give output tiles of 128 x TN for every TN
    (32: orders 2-4; 64, 128, 160, 256: order 5 over 8, 12, 16 and 20
    shells), several row tiles and split-K over the cells; the 30 x 18 x 10
    grid (5400 cells) ends in a partial chunk."""
    g = GridSpec(dims, (0.0, 0.0, 0.0), 1.0, True)
    rng = np.random.default_rng(50 + ns)
    nc = g.n_cells
    w0 = rng.normal(size=nc).astype(np.float32)
    bank = rng.normal(size=(ns, nc)).astype(np.float32)
    w = dict(grid=g, shells=tuple(1.0 + 0.05 * i for i in range(ns)), width=1.0)
    plan = plan_for(w, max_order=5, precision=precision)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((ns, stride), np.float32)
    B[:, :nc] = bank
    for orders in [(2, 3), (4,), (5,), (2, 3, 4, 5)]:
        sums = plan.contract(dev(torch, w0), dev(torch, B), stride, orders=orders)
        for n in orders:
            want, awant = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
            e = normwise(sums[n].cpu().numpy(), want, awant)
            assert e <= SPLIT_TOL[precision], f"order {n}: {e:.3e}"
    plan.close()


@pytest.mark.parametrize("precision", ["split_bf16", "split_fp16"])
def test_split16_dynamic_range(torch, precision):
    """Fields far outside the FP16 range (|W0| ~ 1e3, |W_s| ~ 1e4 on one
    shell and 1e-3 on another, products up to 1e15): the per-factor
    power-of-two scales keep the FP16 operands finite and the split forms
    inside their gates; all-zero shells give exact zeros."""
    g = GridSpec((24, 20, 18), (0.0, 0.0, 0.0), 1.0, True)
    rng = np.random.default_rng(77)
    nc = g.n_cells
    ns = 6
    w0 = (1e3 * rng.normal(size=nc)).astype(np.float32)
    bank = rng.normal(size=(ns, nc))
    bank[0] *= 1e4
    bank[1] *= 1e-3
    bank[2] = 0.0
    bank = bank.astype(np.float32)
    w = dict(grid=g, shells=tuple(1.0 + 0.05 * i for i in range(ns)), width=1.0)
    plan = plan_for(w, max_order=5, precision=precision)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((ns, stride), np.float32)
    B[:, :nc] = bank
    sums = plan.contract(dev(torch, w0), dev(torch, B), stride, orders=(2, 3, 4, 5))
    for n in (2, 3, 4, 5):
        want, awant = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
        got = sums[n].cpu().numpy()
        assert np.all(np.isfinite(got)), f"order {n}"
        assert normwise(got, want, awant) <= SPLIT_TOL[precision], f"order {n}"
        assert np.all(got[awant == 0.0] == 0.0), f"order {n}: zero shells"
    plan.close()


def test_order_subsets(torch, p32, ref32):
    for orders in [(2,), (3,), (4,), (5,), (2, 4), (3, 5)]:
        plan, res = _run(torch, p32, orders, max_order=5)
        _check_sums(res, ref32, 4, orders)
        plan.close()


def test_blocked_contraction_16_shells(torch):
    """16 shells up to order 5 (the blocked kernel) on a small periodic box,
    against the oracle's product sums of the same float32 fields."""
    g = GridSpec((24, 20, 16), (0.0, 0.0, 0.0), 1.0, True)
    rng = np.random.default_rng(5)
    nc = g.n_cells
    w0 = rng.normal(size=nc).astype(np.float32)
    bank = rng.normal(size=(16, nc)).astype(np.float32)
    w = dict(grid=g, shells=tuple(1.0 + 0.1 * i for i in range(16)), width=1.0)
    plan = plan_for(w, max_order=5)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((16, stride), np.float32)
    B[:, :nc] = bank
    for orders in [(2, 3), (4,), (5,), (2, 3, 4, 5)]:
        sums = plan.contract(dev(torch, w0), dev(torch, B), stride, orders=orders)
        for n in orders:
            want, awant = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
            e = normwise(sums[n].cpu().numpy(), want, awant)
            assert e <= TOL, f"order {n}: {e:.3e}"
    plan.close()


def test_reg_contraction_ragged(torch):
    """Register kernel on a cell count that is not a multiple of the chunk or
    of 4 (ragged tail read without bulk copies)."""
    g = GridSpec((10, 12, 6), (0.0, 0.0, 0.0), 1.0, True)  # 720 cells: 3 chunks of 224 + 48
    rng = np.random.default_rng(6)
    nc = g.n_cells
    w = dict(grid=g, shells=tuple(1.0 + 0.1 * i for i in range(16)), width=1.0)
    plan = plan_for(w, max_order=3)
    for count in (nc,):
        w0 = rng.normal(size=count).astype(np.float32)
        bank = rng.normal(size=(16, count)).astype(np.float32)
        sums = plan.contract(dev(torch, w0), dev(torch, bank.reshape(-1)), count, orders=(2, 3))
        for n in (2, 3):
            want, awant = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
            assert normwise(sums[n].cpu().numpy(), want, awant) <= TOL
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
def test_survey_subbox_s16(torch, precision):
    """The 512^3 survey catalog cut to a 64^3 periodic sub-box (12 of its
    shells, orders 2 and 3) against the oracle, in the plain and the mixed
    (fused) form."""
    w = workload("survey512", scale=0.25)
    lo = np.array([-256.0, -256.0, 1300.0])
    def cut(c):
        sel = ((c.x >= lo[0]) & (c.x < lo[0] + 512) & (c.y >= lo[1]) & (c.y < lo[1] + 512)
               & (c.z >= lo[2]) & (c.z < lo[2] + 512))
        return Catalog(c.x[sel] - np.float32(lo[0]), c.y[sel] - np.float32(lo[1]), c.z[sel] - np.float32(lo[2]))
    g = GridSpec((64, 64, 64), (0.0, 0.0, 0.0), 8.0, True)
    sub = dict(grid=g, shells=w["shells"][:12], width=w["width"], data=cut(w["data"]), randoms=cut(w["randoms"]))
    assert sub["data"].n > 1000 and sub["randoms"].n > 100000
    ref = O.correlate(g, sub["shells"], sub["width"], sub["data"], sub["randoms"], orders=(2, 3), engine="fft")
    plan, res = _run(torch, sub, (2, 3), precision=precision)
    assert plan.fused is (precision == "split_tf32")
    _check_sums(res, ref, len(sub["shells"]), (2, 3))
    plan.close()


# ---------------------------------------------------------------------------
# behaviour

def test_determinism_and_host_io(torch, p32):
    plan = plan_for(p32, max_order=5)
    plan.set_randoms(*dev_cat(torch, p32["randoms"]))
    a = plan.compute(*dev_cat(torch, p32["data"]), orders=(2, 3, 4, 5), out="host")
    b = plan.compute(*dev_cat(torch, p32["data"]), orders=(2, 3, 4, 5), out="host")
    d = p32["data"]
    c = plan.compute(d.x, d.y, d.z, orders=(2, 3, 4, 5), out="host")  # host positions
    for n in (2, 3, 4, 5):
        assert np.array_equal(a["num"][n].numpy(), b["num"][n].numpy())
        assert np.array_equal(a["num"][n].numpy(), c["num"][n].numpy())
    plan.close()


def test_errors(torch, p32):
    from paper_2108_00015_gb300 import CkError
    plan = plan_for(p32)
    d = dev_cat(torch, p32["data"])
    with pytest.raises(CkError) as e:
        plan.compute(*d, orders=(2,))
    assert e.value.code == 11  # no randoms yet
    # randoms in a single cell: B_s = 0 wherever Rt != 0, so den = 0 up to FFT
    # rounding; entries with den <= 0 must be NaN and flagged
    one = Catalog(np.full(10, 155.0, np.float32), np.full(10, 155.0, np.float32), np.full(10, 155.0, np.float32))
    plan.set_randoms(*dev_cat(torch, one))
    res = plan.compute(*d, orders=(2, 3), out="host")
    den = res["den"][2].numpy()
    xi = res["xi"][2].numpy()
    alpha = p32["data"].n / 10.0
    # a single occupied cell gives den_raw = 0; compare with R^2 |O_s| = 100 |O_s|
    assert np.all(np.abs(den) / (alpha ** 2 * 100.0 * np.array(plan.shell_size)) < 1e-4)
    assert np.array_equal(np.isnan(xi), den <= 0)
    assert (res["status"] == 7) == bool((den <= 0).any() or (res["den"][3].numpy() <= 0).any())
    with pytest.raises(CkError):
        plan.compute(*d, orders=(6,))
    plan.close()


def test_guard_band(torch):
    g = GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, False)
    dat = uniform_box(1, 2000, 320.0)
    w = dict(grid=g, shells=(20.0, 40.0), width=10.0, data=dat, randoms=dat)
    plan = plan_for(w)
    plan.set_randoms(*dev_cat(torch, dat))
    from paper_2108_00015_gb300 import CkError
    with pytest.raises(CkError) as e:
        plan.compute(*dev_cat(torch, dat), orders=(2,), out="host")
    assert e.value.code == 6
    plan.close()
