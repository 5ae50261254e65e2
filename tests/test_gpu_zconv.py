"""The z step of the convolution by the shells' short filters (Sec. 2.4's
convolution along z as the sum over the planes a shell reaches, after the
x and y transforms), against the FP64 oracle's convolutions and the
transform route:

- a periodic box filled by the catalog (taps wrap around the z axis), 11
  shells in two groups of 8 with different reaches, and an odd z length;
- a catalog confined to a sub-box of 512 x 512 planes after a wider one, so
  that the planes of the resident spectrum outside the new box still hold
  the old catalog (the pruned forward passes skip them): the sums, and the
  whole-grid W_s that ck_get_bank recomputes, must ignore them;
- single shells on either side of a group boundary, recomputed on request;
- the route's limit: shells reaching more than 31 planes keep the
  transform route.
Tolerances: banks within 1e-5 of max |W| of the oracle's, sums normwise
within 1e-5 of the oracle's (as in the other parity tests)."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _check_sums(res, ref, ns, tol=TOL):
    for n in (2, 3):
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
            e = normwise(got, want, scale)
            assert e <= tol, f"order {n} {key}: normwise error {e:.3e}"


def _bank_close(got, want, what):
    got = np.asarray(got, np.float64)
    e = np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)
    assert e <= TOL, f"{what}: {e:.3e}"


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
def test_direct_filter_periodic_wrap(precision):
    torch = cuda_torch()
    n = (24, 40, 36)
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, True)
    L = tuple(float(v) for v in n)
    shells = tuple(1.0 + 0.55 * i for i in range(11))  # reaches 2 .. 7 planes
    w = dict(grid=g, shells=shells, width=1.0, data=neyman_scott_box(71, 300, 10, 1.5, L),
             randoms=uniform_box(72, 60_000, L))
    plan = plan_for(w, max_order=3, precision=precision)
    assert plan.tuning()["z_direct"] == 1
    ref = O.correlate(g, shells, 1.0, w["data"], w["randoms"], orders=(2, 3), engine="direct")
    banks = {}
    for zd in (1, 0):
        plan.set_tuning(z_direct=zd)
        assert plan.tuning()["z_direct"] == zd
        plan.set_randoms(*dev_cat(torch, w["randoms"]))
        res = plan.compute(*dev_cat(torch, w["data"]), orders=(2, 3), out="host")
        assert res["status"] == 0
        _check_sums(res, ref, len(shells))
        N = plan.field(0).cpu().numpy().astype(np.float64)
        banks[zd] = [plan.bank(s).cpu().numpy() for s in range(len(shells))]
        for s, rad in enumerate(shells):
            want = O.convolve_direct(N, O.shell_offsets(rad, 1.0, 1.0), True)
            _bank_close(banks[zd][s], want, f"z_direct {zd} shell {s}")
    plan.close()


def _confined(n, lo, hi, nd_par, nr, seed):
    lo = np.array(lo, np.float64)
    span = np.array(hi, np.float64) - lo
    d = neyman_scott_box(seed, nd_par, 8, 1.2, tuple(span))
    r = uniform_box(seed + 1, nr, tuple(span))

    def shift(c):
        return Catalog(*(np.asarray(v, np.float64) + lo[a] for a, v in enumerate((c.x, c.y, c.z))))

    def f32(c):
        return Catalog(*(np.asarray(v, np.float32) for v in (c.x, c.y, c.z)))
    return f32(shift(d)), f32(shift(r))


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
def test_direct_filter_ignores_stale_planes(precision):
    torch = cuda_torch()
    n = (32, 512, 512)
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, False)
    shells = (1.5, 2.5, 3.5, 4.5)
    # a wider catalog first: its transformed planes stay in the spectrum
    wide_d, wide_r = _confined(n, (5, 40, 60), (27, 470, 450), 600, 200_000, 80)
    data, rand = _confined(n, (6, 120, 200), (26, 330, 331), 400, 120_000, 90)
    plan = plan_for(dict(grid=g, shells=shells, width=1.0), max_order=3, precision=precision)
    assert plan.tuning()["z_direct"] == 1
    plan.set_randoms(*dev_cat(torch, wide_r))
    plan.compute(*dev_cat(torch, wide_d), orders=(2, 3), out="host")
    plan.set_randoms(*dev_cat(torch, rand))
    res = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
    assert res["status"] == 0
    ref = O.correlate(g, shells, 1.0, data, rand, orders=(2, 3), engine="fft")
    _check_sums(res, ref, len(shells))
    N = plan.field(0).cpu().numpy().astype(np.float64)
    for s, rad in enumerate(shells):
        want = O.convolve_fft(N, O.shell_offsets(rad, 1.0, 1.0))
        _bank_close(plan.bank(s).cpu().numpy(), want, f"shell {s}")
    plan.close()


def test_direct_filter_single_shells_across_groups():
    torch = cuda_torch()
    n = (20, 24, 30)
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, True)
    L = tuple(float(v) for v in n)
    shells = tuple(1.0 + 0.18 * i for i in range(19))  # groups of 8, 8 and 3
    w = dict(grid=g, shells=shells, width=0.5, data=neyman_scott_box(73, 200, 10, 1.5, L),
             randoms=uniform_box(74, 30_000, L))
    plan = plan_for(w, max_order=2, precision="fp32")
    assert plan.tuning()["z_direct"] == 1
    plan.set_randoms(*dev_cat(torch, w["randoms"]))
    res = plan.compute(*dev_cat(torch, w["data"]), orders=(2,), out="host")
    assert res["status"] == 0
    N = plan.field(0).cpu().numpy().astype(np.float64)
    for s in (0, 7, 8, 15, 16, 18):
        want = O.convolve_direct(N, O.shell_offsets(shells[s], 0.5, 1.0), True)
        _bank_close(plan.bank(s).cpu().numpy(), want, f"shell {s}")
    plan.close()


@pytest.mark.parametrize("radius,direct", [(30.0, 1), (32.0, 0)])
def test_direct_filter_reach_limit(radius, direct):
    cuda_torch()
    g = GridSpec((72, 72, 72), (0.0, 0.0, 0.0), 1.0, True)
    plan = plan_for(dict(grid=g, shells=(radius,), width=1.0), max_order=2, precision="fp32")
    assert plan.tuning()["z_direct"] == direct
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
def test_empty_catalogs_on_pruned_grid(precision):
    """An empty catalog, or one whose points all fall outside the box, has
    an empty support box (stored as lo > hi): every pass, pruned or not, and
    either z route visits nothing, the call reports CK_ERR_EMPTY_CATALOG,
    and the plan then serves the next catalog exactly as a new one would."""
    from paper_2108_00015_gb300 import CkError
    torch = cuda_torch()
    n = (32, 512, 512)
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, False)
    shells = (1.5, 2.5, 3.5)
    data, rand = _confined(n, (6, 120, 200), (26, 330, 331), 300, 80_000, 95)
    ref = O.correlate(g, shells, 1.0, data, rand, orders=(2, 3), engine="fft")
    empty = Catalog(*(np.zeros(0, np.float32) for _ in range(3)))
    outside = Catalog(*(np.full(50, -5.0, np.float32) for _ in range(3)))
    plan = plan_for(dict(grid=g, shells=shells, width=1.0), max_order=3, precision=precision)
    for zd in (1, 0):
        plan.set_tuning(z_direct=zd)
        for bad in (empty, outside):
            try:
                plan.set_randoms(*dev_cat(torch, bad))
            except CkError as e:
                assert e.code == 12
            plan.set_randoms(*dev_cat(torch, rand))
            with pytest.raises(CkError) as e:
                plan.compute(*dev_cat(torch, bad), orders=(2, 3), out="host")
            assert e.value.code == 12
            res = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
            assert res["status"] == 0
            _check_sums(res, ref, len(shells))
    plan.close()
