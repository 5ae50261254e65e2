"""The fused pass visits only the box of occupied cells (W_0 = N or Rt
vanishes outside it, so the sums of Eq. 11 do too): catalogs confined to a
sub-box of a survey box, against the FP64 oracle over every cell.  Covers
the 512-point y and z passes (planes and rows outside the box skipped), the
register x pass with several grid rows per tile (8 shells, half-length 16)
and with one (5 shells, half-length 32), the shared-memory x pass of an odd
half-length, and the plain path (no pruning) on the same catalog."""
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
        plan.set_randoms(*dev_cat(torch, rand))
        res = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
        assert res["status"] == 0
        _check(res, ref, ns)
        plan.close()
