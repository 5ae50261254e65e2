"""The fused pass visits only the box of occupied cells (W_0 = N or Rt
vanishes outside it, so the sums of Eq. 11 do too): catalogs confined to a
sub-box of a survey box, against the FP64 oracle over every cell.  Covers
the 512-point y and z passes (planes and rows outside the box skipped), the
register x pass with several grid rows per tile (8 shells, half-length 16)
and with one (5 shells, half-length 32), the shared-memory x pass of an odd
half-length, and the plain path (no pruning) on the same catalog, each
with the z step by the shells' short filters and by the K^ z pass."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _confined(n, lo, hi, nd_par, nr, seed):
    """Clustered data and uniform randoms inside the cells lo..hi-1 of a
    unit-cell box of n cells per axis."""
    lo = np.array(lo, np.float64)
    span = np.array(hi, np.float64) - lo
    d = neyman_scott_box(seed, nd_par, 8, 1.2, tuple(span))
    r = uniform_box(seed + 1, nr, tuple(span))
    def shift(c):
        return Catalog(*(np.asarray(v, np.float64) + lo[a] for a, v in enumerate((c.x, c.y, c.z))))
    def f32(c):
        return Catalog(*(np.asarray(v, np.float32) for v in (c.x, c.y, c.z)))
    return f32(shift(d)), f32(shift(r))


def _check(res, ref, ns):
    for n in (2, 3):
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
            e = normwise(got, want, scale)
            assert e <= TOL, f"order {n} {key}: normwise error {e:.3e}"


@pytest.mark.parametrize("n,lo,hi,shells", [
    ((32, 512, 512), (6, 120, 200), (26, 330, 331), tuple(1.0 + 0.6 * i for i in range(8))),  # 512-point y, z
    ((30, 40, 36), (8, 9, 10), (22, 30, 26), (1.5, 2.5, 3.5)),                       # x half-length 15
    ((64, 48, 40), (10, 12, 9), (50, 34, 30), (1.5, 2.5, 3.5, 5.0, 6.0)),            # register x, M = 32
])
def test_fused_support_box(n, lo, hi, shells):
    torch = cuda_torch()
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, False)
    data, rand = _confined(n, lo, hi, 400, 120_000, sum(n))
    w = dict(grid=g, shells=shells, width=1.0, data=data, randoms=rand)
    ref = O.correlate(g, shells, 1.0, data, rand, orders=(2, 3), engine="fft")
    ns = len(shells)
    for prec in ("split_tf32", "fp32"):
        plan = plan_for(w, max_order=3, precision=prec)
        assert plan.fused is (prec == "split_tf32")
        for zd in (1, 0):  # the z step by the short filters, then by the K^ z pass
            plan.set_tuning(z_direct=zd)
            plan.set_randoms(*dev_cat(torch, rand))
            res = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
            assert res["status"] == 0
            _check(res, ref, ns)
        plan.close()


@pytest.mark.parametrize("precision", ["split_tf32", "fp32"])
def test_field_exact_across_catalogs(precision):
    """The preparations rewrite only the planes of the occupied box and of
    the previous occupied box: on one plan, catalogs confined to different
    sub-boxes (and a continuous field loaded in between, which may be
    nonzero anywhere) leave a field buffer that is N (or R) on every cell,
    exactly zero where both histograms are, count buffers equal to the
    oracle's histograms, and sums that match the oracle's."""
    torch = cuda_torch()
    n = (30, 40, 36)
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, False)
    shells = (1.5, 2.5, 3.5)
    boxes = [((8, 9, 4), (22, 30, 14)), ((6, 8, 20), (24, 31, 31)), ((9, 10, 12), (21, 29, 24))]
    cats = [_confined(n, lo, hi, 300, 60_000, 7 + i) for i, (lo, hi) in enumerate(boxes)]
    w = dict(grid=g, shells=shells, width=1.0, data=cats[0][0], randoms=cats[0][1])
    plan = plan_for(w, max_order=3, precision=precision)

    def check_field(which, D, R):
        # which = 0: N = D - alpha R; which = 1: R as float (before alpha)
        f = plan.field(which).cpu().numpy().astype(np.float64)
        _, N, _ = O.density_fields(D, R)
        want = N if which == 0 else R.astype(np.float64)
        empty = (D == 0) & (R == 0) if which == 0 else (R == 0)
        assert np.all(f[empty] == 0.0)
        assert np.max(np.abs(f - want)) <= 1e-6 * max(1.0, np.max(np.abs(want)))

    rng = np.random.default_rng(5)
    for i, (data, rand) in enumerate(cats):
        if i == 2:  # first a continuous field over more planes than this catalog's box
            d = np.zeros((n[2], n[1], n[0]), np.float32)
            d[5:-5, 5:-5, 5:-5] = rng.uniform(0.5, 1.5, (n[2] - 10, n[1] - 10, n[0] - 10))
            plan.compute_continuous(torch.from_numpy(d).cuda(), None, orders=(2,), out="host")
        D, _ = O.grid_counts(data.x, data.y, data.z, g)
        R, _ = O.grid_counts(rand.x, rand.y, rand.z, g)
        plan.set_randoms(*dev_cat(torch, rand))
        check_field(1, D, R)
        res = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
        assert res["status"] == 0
        check_field(0, D, R)
        # the count buffers, cleared only where the previous histograms were
        # (everywhere after the continuous field used the data buffer)
        gd, gr = plan.grids()
        assert np.array_equal(gd.cpu().numpy().astype(np.uint32), D)
        assert np.array_equal(gr.cpu().numpy().astype(np.uint32), R)
        ref = O.correlate(g, shells, 1.0, data, rand, orders=(2, 3), engine="fft")
        _check(res, ref, len(shells))
        # the whole W_s on request (the plan's own bank covers only the box's planes)
        _, N, _ = O.density_fields(D, R)
        for k, rad in enumerate(shells):
            want = O.convolve_direct(N, O.shell_offsets(rad, 1.0, 1.0), False)
            got = plan.bank(k).cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, np.max(np.abs(want))), (i, k)
    plan.close()


@pytest.mark.parametrize("precision", ["split_tf32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("n,lo,hi,cube", [((30, 40, 36), (8, 9, 16), (22, 30, 26), (6, 10, 5)),
                                          ((24, 512, 512), (4, 150, 220), (20, 330, 300), (6, 160, 100))])
def test_bank_planes_higher_orders(n, lo, hi, cube, precision):
    """Plans that keep the bank (orders up to 4, split forms on the tensor
    cores) transform and sum only the occupied planes.  A first catalog
    packs 2M points into a small cube on other planes, leaving W_s of about
    1e6 in the bank's planes outside the next catalog's box; a sparse
    catalog confined to that box must then give sums of every order within
    the form's gate of the oracle's, so nothing (the FP16 row scales
    included) reads those planes."""
    torch = cuda_torch()
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, False)
    shells = (1.5, 2.5, 3.5)
    w = dict(grid=g, shells=shells, width=1.0)
    plan = plan_for(w, max_order=4, precision=precision)
    assert not plan.fused
    rng = np.random.default_rng(31)
    c0 = np.array(cube, np.float64)
    packed = Catalog(*(np.asarray(c0[a] + rng.uniform(0.0, 4.0, 2_000_000), np.float32) for a in range(3)))
    spread = Catalog(*(np.asarray(rng.uniform(5.0, n[a] - 5.0, 200_000), np.float32) for a in range(3)))
    plan.set_randoms(*dev_cat(torch, spread))
    plan.compute(*dev_cat(torch, packed), orders=(2, 3, 4), out="host")
    data, rand = _confined(n, lo, hi, 300, 80_000, 11)
    ref = O.correlate(g, shells, 1.0, data, rand, orders=(2, 3, 4), engine="fft")
    plan.set_randoms(*dev_cat(torch, rand))
    res = plan.compute(*dev_cat(torch, data), orders=(2, 3, 4), out="host")
    assert res["status"] == 0
    tol = 5e-5 if precision == "split_bf16" else TOL
    for order in (2, 3, 4):
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            want = O.dense_tensor(ref[f"{key}{order}"], len(shells), order - 1)
            scale = O.dense_tensor(ref[f"{akey}{order}"], len(shells), order - 1)
            assert normwise(res[key][order].numpy(), want, scale) <= tol, (order, key)
    plan.close()
