"""Weighted histograms (ck_set_randoms_weighted / ck_compute_weighted;
Sec. 2.2 weighted counts, Sec. 3 systematic and FKP weights): the gridded
cells bit-exact against the oracle's grid_weights (each weight rounded to a
multiple of 2^-32, exact sums, rounded to float32), with signed and
non-finite weights and points outside a survey box; the product sums
against the oracle's weighted correlation; unit weights bit-identical to the
unweighted path; host weights through the staging path."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _box(seed, periodic=True):
    g = GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, periodic)
    data = neyman_scott_box(seed, 250, 12, 12.0, 320.0)
    rand = uniform_box(seed + 1, 30000, 320.0)
    return g, data, rand


def _weights(seed, n, signed=False, bad=False):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.2, 1.8, n).astype(np.float32)  # FKP-like: 1 / (1 + n P) in (0, 1], systematics ~ 1
    if signed:
        w[::7] *= -0.5
    if bad:
        w[3] = np.nan
        w[10] = np.inf
    return w


def test_weighted_grids_bit_exact(torch):
    # a survey box with points outside it, signed and non-finite weights
    g = GridSpec((30, 24, 20), (5.0, -3.0, 1.0), 8.0, False)
    L = np.array(g.n, np.float64) * g.cell
    c = uniform_box(3, 20000, tuple(L + 16.0))
    cat = Catalog((c.x - 8.0 + 5.0).astype(np.float32), (c.y - 8.0 - 3.0).astype(np.float32),
                  (c.z - 8.0 + 1.0).astype(np.float32))
    wd = _weights(5, cat.n, signed=True, bad=True)
    wr = _weights(6, cat.n)
    w = dict(grid=g, shells=(16.0, 24.0), width=8.0)
    plan = plan_for(w, max_order=2)
    x, y, z = dev_cat(torch, cat)
    plan.set_randoms(x, y, z, w=dev(torch, wr))
    from paper_2108_00015_gb300 import CkError
    try:
        res = plan.compute(x, y, z, orders=(2,), out="host", w=dev(torch, wd))
        dropped = res["dropped"].numpy().tolist()
    except CkError:  # the points fill the box: the survey box reports its guard band
        dropped = None
    D, R = plan.grids()
    Dw, _, dd = O.grid_weights(cat.x, cat.y, cat.z, wd, g)
    Rw, _, dr = O.grid_weights(cat.x, cat.y, cat.z, wr, g)
    got_d = D.cpu().numpy().view(np.float32)
    got_r = R.cpu().numpy().view(np.float32)
    assert np.array_equal(got_d, Dw.astype(np.float32))
    assert np.array_equal(got_r, Rw.astype(np.float32))
    if dropped is not None:
        assert dropped == [dd, dr]
    plan.close()


@pytest.mark.parametrize("precision,max_order,orders", [
    ("fp32", 3, (2, 3)), ("split_tf32", 3, (2, 3)), ("split_tf32", 4, (2, 3, 4))])
def test_weighted_sums_vs_oracle(torch, precision, max_order, orders):
    g, data, rand = _box(21)
    wd = _weights(7, data.n)
    wr = _weights(8, rand.n)
    shells = (20.0, 35.0, 50.0)
    ref = O.correlate(g, shells, 10.0, data, rand, orders=orders, engine="fft", data_weights=wd,
                      random_weights=wr)
    plan = plan_for(dict(grid=g, shells=shells, width=10.0), max_order=max_order, precision=precision)
    plan.set_randoms(*dev_cat(torch, rand), w=dev(torch, wr))
    res = plan.compute(*dev_cat(torch, data), orders=orders, out="host", w=dev(torch, wd))
    for n in orders:
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], len(shells), n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], len(shells), n - 1)
            e = normwise(got, want, scale)
            assert e <= TOL, f"order {n} {key}: {e:.3e}"
    plan.close()


def test_unit_weights_match_counts(torch):
    """Weights of 1 give the unweighted path's results bit for bit (the cells
    are exact integer counts and alpha the same ratio); weighted data over
    unweighted randoms mixes the two kinds of field."""
    g, data, rand = _box(31)
    plan = plan_for(dict(grid=g, shells=(20.0, 35.0), width=10.0), max_order=3, precision="split_tf32")
    d = dev_cat(torch, data)
    plan.set_randoms(*dev_cat(torch, rand))
    plain = plan.compute(*d, orders=(2, 3), out="host")
    ones = torch.ones(data.n, dtype=torch.float32, device="cuda")
    mixed = plan.compute(*d, orders=(2, 3), out="host", w=ones)
    plan.set_randoms(*dev_cat(torch, rand), w=torch.ones(rand.n, dtype=torch.float32, device="cuda"))
    both = plan.compute(*d, orders=(2, 3), out="host", w=ones)
    for n in (2, 3):
        for key in ("xi", "num", "den"):
            assert np.array_equal(plain[key][n].numpy(), mixed[key][n].numpy()), (n, key)
            assert np.array_equal(plain[key][n].numpy(), both[key][n].numpy()), (n, key)
    plan.close()


def test_host_weights(torch):
    """Host positions and weights go through the staging slots (more points
    than one slot holds) and give the device path's results."""
    g = GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, True)
    rand = uniform_box(41, 2_500_000, 320.0)
    data = neyman_scott_box(42, 400, 10, 12.0, 320.0)
    wr = _weights(43, rand.n)
    wd = _weights(44, data.n)
    plan = plan_for(dict(grid=g, shells=(20.0, 35.0), width=10.0), max_order=2)
    plan.set_randoms(rand.x, rand.y, rand.z, w=wr)
    host = plan.compute(data.x, data.y, data.z, orders=(2,), out="host", w=wd)
    Rh = plan.grids()[1].cpu().numpy()
    plan.set_randoms(*dev_cat(torch, rand), w=dev(torch, wr))
    devr = plan.compute(*dev_cat(torch, data), orders=(2,), out="host", w=dev(torch, wd))
    Rd = plan.grids()[1].cpu().numpy()
    assert np.array_equal(Rh, Rd)
    for key in ("xi", "num", "den"):
        assert np.array_equal(host[key][2].numpy(), devr[key][2].numpy())
    plan.close()


def test_pinned_host_positions(torch):
    """Page-locked host positions (and weights) are read in place by the
    gridding kernel: the same grids and sums as the device and staged paths."""
    g = GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, True)
    rand = uniform_box(61, 3_000_000, 320.0)
    data = neyman_scott_box(62, 400, 10, 12.0, 320.0)
    wr = _weights(63, rand.n)

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    plan = plan_for(dict(grid=g, shells=(20.0, 35.0), width=10.0), max_order=3)
    for w in (None, wr):
        plan.set_randoms(*dev_cat(torch, rand), w=None if w is None else dev(torch, w))
        want = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
        Rd = plan.grids()[1].cpu().numpy()
        # the pinned arrays are read after the calls return: keep them alive
        hr = [pinned(rand.x), pinned(rand.y), pinned(rand.z)]
        hw = None if w is None else pinned(w)
        hd = [pinned(data.x), pinned(data.y), pinned(data.z)]
        plan.set_randoms(*hr, w=hw)
        got = plan.compute(*hd, orders=(2, 3), out="host")
        assert np.array_equal(plan.grids()[1].cpu().numpy(), Rd)
        for n in (2, 3):
            for key in ("xi", "num", "den"):
                assert np.array_equal(got[key][n].numpy(), want[key][n].numpy()), (w is None, n, key)
    plan.close()


@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_gridding_alignment_and_tails(torch, offset):
    """Coordinate and weight arrays that start 0..3 elements into a device
    buffer (16-byte aligned or not) and point counts that are not multiples
    of four: the 16-byte load path, the element path and the tail give
    counts and weight sums bit-identical to the oracle's."""
    g = GridSpec((30, 24, 20), (5.0, -3.0, 1.0), 8.0, True)
    L = np.array(g.n, np.float64) * g.cell
    n = 20003 + 5 * offset  # never a multiple of four: every path has a tail
    c = uniform_box(11 + offset, n, tuple(L))
    cat = Catalog((c.x + 5.0).astype(np.float32), (c.y - 3.0).astype(np.float32), (c.z + 1.0).astype(np.float32))
    wts = _weights(12 + offset, n, signed=True, bad=True)

    def shifted(a):
        buf = torch.zeros(n + 3, dtype=torch.float32, device="cuda")
        buf[offset:offset + n] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        return buf[offset:offset + n]

    x, y, z, w = (shifted(a) for a in (cat.x, cat.y, cat.z, wts))
    assert (x.data_ptr() % 16 == 0) == (offset == 0)
    plan = plan_for(dict(grid=g, shells=(16.0,), width=8.0), max_order=2)
    plan.set_randoms(x, y, z)
    res = plan.compute(x, y, z, orders=(2,), out="host", w=w)
    D, R = plan.grids()
    want, wdrop = O.grid_counts(cat.x, cat.y, cat.z, g)
    assert np.array_equal(R.cpu().numpy().astype(np.uint32), want)
    Dw, _, dd = O.grid_weights(cat.x, cat.y, cat.z, wts, g)
    assert np.array_equal(D.cpu().numpy().view(np.float32), Dw.astype(np.float32))
    assert res["dropped"].numpy().tolist() == [dd, wdrop]
    plan.close()
