"""A survey box cut into z slabs on one device (the single-GPU emulation of
the domain decomposition): each slab is a zero-padded plan over its owned
planes plus a halo of max|m_z| planes (ck_plan_set_region with the whole
catalog's alpha); the slabs' num and den summed must equal the undivided
plan's and the FP64 oracle's (Eq. 19), for 2 and 3 slabs, in the plain and
the mixed form.  The same decomposition over gloo ranks is tested on CPU."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from paper_2108_00015_gb300.parallel import in_planes, slab_box, slab_planes
from synth import Catalog, GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev_cat, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-5
SHELLS = (1.5, 2.5, 3.5, 4.5)


@pytest.fixture(scope="module")
def case():
    g = GridSpec((40, 36, 60), (0.0, 0.0, 0.0), 1.0, False)
    span = (32.0, 28.0, 52.0)
    def inside(c):
        return Catalog(*(np.asarray(v, np.float32) + np.float32(4.0) for v in (c.x, c.y, c.z)))
    data = inside(neyman_scott_box(5, 300, 10, 1.5, span))
    rand = inside(uniform_box(6, 150_000, span))
    ref = O.correlate(g, SHELLS, 1.0, data, rand, orders=(2, 3), engine="fft")
    return g, data, rand, ref


def _plan(n, origin, precision):
    from paper_2108_00015_gb300 import Plan
    return Plan(n, origin, 1.0, False, SHELLS, 1.0, max_order=3, precision=precision, padded=True)


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
@pytest.mark.parametrize("parts", [2, 3])
def test_slabs_add_up(case, parts, precision):
    torch = cuda_torch()
    g, data, rand, ref = case
    nz = g.n[2]
    alpha = data.n / rand.n  # every point lies in the box
    whole = _plan(g.n, g.origin, precision)
    halo = whole.max_offset[2]
    whole.set_randoms(*dev_cat(torch, rand))
    wres = whole.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
    whole.close()
    num = {n: 0.0 for n in (2, 3)}
    den = {n: 0.0 for n in (2, 3)}
    for rank in range(parts):
        z0, z1 = slab_planes(nz, parts, rank)
        lo, hi = slab_box(nz, z0, z1, halo)
        pick = lambda c: Catalog(*(v[in_planes(c.z, g.origin[2], g.cell, lo, hi)] for v in (c.x, c.y, c.z)))  # noqa: E731
        p = _plan((g.n[0], g.n[1], hi - lo), (g.origin[0], g.origin[1], g.origin[2] + lo * g.cell), precision)
        p.set_region(z0 - lo, z1 - lo, alpha)
        p.set_randoms(*dev_cat(torch, pick(rand)))
        r = p.compute(*dev_cat(torch, pick(data)), orders=(2, 3), out="host")
        assert r["status"] == 0
        for n in (2, 3):
            num[n] = num[n] + r["num"][n].numpy()
            den[n] = den[n] + r["den"][n].numpy()
        p.close()
    ns = len(SHELLS)
    for n in (2, 3):
        for key, got, akey in (("num", num[n], "abs_num"), ("den", den[n], "abs_den")):
            want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
            assert normwise(got, want, scale) <= TOL, f"{parts} slabs, order {n} {key} vs oracle"
            assert normwise(got, wres[key][n].numpy(), scale) <= 2 * TOL, f"{parts} slabs, order {n} {key} vs whole"
