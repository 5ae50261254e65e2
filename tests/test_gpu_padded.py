"""Survey boxes transformed on a zero-padded grid (CK_GRID_PADDED): the
occupied cells reach the box faces, which a plan on the box itself reports
as a guard-band violation (CK_ERR_GUARD_BAND, 6); the padded plan gives the
linear (zero outside the box) convolution of the oracle's direct engine,
for box sizes that need not be transform lengths (odd, prime factors 17,
23), points outside the box dropped and counted."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, uniform_box
from tests.gpu_util import cuda_torch, dev_cat, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _plan(g, shells, width, max_order, precision, padded):
    from paper_2108_00015_gb300 import Plan
    return Plan(g.n, g.origin, g.cell, False, shells, width, max_order=max_order, precision=precision,
                padded=padded)


def _catalogs(g, seed, nd, nr):
    """Uniform points over the box and a margin of one cell around it, so
    that the occupied cells touch every face and some points fall outside."""
    L = np.array(g.n, np.float64) * g.cell
    o = np.array(g.origin, np.float64) - g.cell

    def cat(s, n):
        c = uniform_box(s, n, tuple(L + 2 * g.cell))
        return Catalog((c.x + o[0]).astype(np.float32), (c.y + o[1]).astype(np.float32),
                       (c.z + o[2]).astype(np.float32))
    return cat(seed, nd), cat(seed + 1, nr)


def _check(res, ref, ns, orders):
    for n in orders:
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
            e = normwise(got, want, scale)
            assert e <= TOL, f"order {n} {key}: {e:.3e}"


@pytest.mark.parametrize("precision,orders", [("fp32", (2, 3)), ("split_tf32", (2, 3)), ("fp32", (2, 3, 4))])
def test_padded_matches_linear_convolution(torch, precision, orders):
    from paper_2108_00015_gb300 import CkError
    g = GridSpec((24, 20, 18), (0.0, 0.0, 0.0), 10.0, False)
    shells, width = (20.0, 30.0, 40.0), 10.0
    dat, ran = _catalogs(g, 3, 3000, 20000)
    ref = O.correlate(g, shells, width, dat, ran, orders=orders, engine="direct")
    # on the box itself the kernel reach wraps: the plan reports it
    box = _plan(g, shells, width, max(orders), precision, padded=False)
    box.set_randoms(*dev_cat(torch, ran))
    with pytest.raises(CkError) as e:
        box.compute(*dev_cat(torch, dat), orders=orders, out="host")
    assert e.value.code == 6
    box.close()
    plan = _plan(g, shells, width, max(orders), precision, padded=True)
    for a in range(3):
        assert plan.fft_n[a] >= g.n[a] + plan.max_offset[a] and plan.fft_n[a] % 2 == 0
    plan.set_randoms(*dev_cat(torch, ran))
    res = plan.compute(*dev_cat(torch, dat), orders=orders, out="host")
    assert res["status"] == 0
    _check(res, ref, len(shells), orders)
    assert res["dropped"].numpy().tolist() == [ref["dropped_d"], ref["dropped_r"]]
    plan.close()


def test_padded_odd_box(torch):
    """A 23 x 17 x 15 box (odd sizes, not transform lengths) with orders up to 4."""
    g = GridSpec((23, 17, 15), (5.0, -3.0, 2.0), 8.0, False)
    shells, width = (16.0, 24.0, 32.0), 8.0
    dat, ran = _catalogs(g, 11, 2500, 15000)
    ref = O.correlate(g, shells, width, dat, ran, orders=(2, 3, 4), engine="direct")
    plan = _plan(g, shells, width, 4, "fp32", padded=True)
    plan.set_randoms(*dev_cat(torch, ran))
    res = plan.compute(*dev_cat(torch, dat), orders=(2, 3, 4), out="host")
    _check(res, ref, len(shells), (2, 3, 4))
    D, R = plan.grids()
    # the box's counts sit in the corner of the padded grid; the padding is empty
    nz, ny, nx = g.n[2], g.n[1], g.n[0]
    assert np.array_equal(D.cpu().numpy()[:nz, :ny, :nx], ref["D"])
    assert int(D.sum()) == int(ref["D"].sum()) and int(R.sum()) == int(ref["R"].sum())
    plan.close()
