"""Fields on the grid and per-cell maps (Secs. 2.7, 2.8, 4.2):

* ck_compute_continuous (Eqs. 15-17): the over-density of two continuous
  maps and its plain sums, against the oracle's delta_field + field_sums;
  delta given directly (r NULL);
* ck_compute_cross (Sec. 2.8): two different maps, W_0 = f0 and
  W_s = f1 *** K_s, on a padded box (linear convolution) and on a box plan
  (guard band reported);
* host fields through the staging path, bit-identical to device fields;
* ck_product_map: W_0 W_s / <B_0 B_s> per cell against the oracle's
  product_map (normwise in the terms of W_s), and its sum rule against the
  same compute's num_2; errors when no catalog compute precedes it.
"""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec, continuous_maps, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev, dev_cat, normwise

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _plan(g, shells, width, max_order, precision, padded=False):
    from paper_2108_00015_gb300 import Plan
    return Plan(g.n, g.origin, g.cell, g.periodic, shells, width, max_order=max_order, precision=precision,
                padded=padded)


def _check(res, ref, ns, orders):
    for n in orders:
        got = res["num"][n].cpu().numpy()
        want = O.dense_tensor(ref[f"num{n}"], ns, n - 1)
        scale = O.dense_tensor(ref[f"abs_num{n}"], ns, n - 1)
        e = normwise(got, want, scale)
        assert e <= TOL, f"order {n}: {e:.3e}"
        assert np.array_equal(res["xi"][n].cpu().numpy(), got)
        assert np.all(res["den"][n].cpu().numpy() == 1.0)


@pytest.mark.parametrize("precision,orders", [("fp32", (2, 3)), ("split_tf32", (2, 3)), ("fp32", (2, 3, 4)),
                                              ("split_tf32", (2, 3, 4))])
def test_continuous_vs_oracle(torch, precision, orders):
    g = GridSpec((32, 30, 24), (0.0, 0.0, 0.0), 10.0, True)
    shells, width = (20.0, 35.0, 50.0), 10.0
    D, R = continuous_maps(3, (24, 30, 32), g.cell)
    delta = O.delta_field(D, R)
    ref = O.field_sums(g, shells, width, delta, delta, orders=orders, engine="fft")
    plan = _plan(g, shells, width, max(orders), precision)
    res = plan.compute_continuous(dev(torch, D), dev(torch, R), orders=orders, out="host")
    _check(res, ref, len(shells), orders)
    # the loaded field is delta (float32 of the FP64 value, within 2 roundings)
    got = plan.field(0).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - delta) <= 2.5e-7 * np.abs(delta) + 1e-30)
    # delta given directly
    res2 = plan.compute_continuous(dev(torch, delta.astype(np.float32)), None, orders=orders, out="host")
    for n in orders:
        e = normwise(res2["num"][n].numpy(), O.dense_tensor(ref[f"num{n}"], len(shells), n - 1),
                     O.dense_tensor(ref[f"abs_num{n}"], len(shells), n - 1))
        assert e <= TOL
    plan.close()


def _two_maps(g, seed):
    D0, R0 = continuous_maps(seed, (g.n[2], g.n[1], g.n[0]), g.cell, footprint=2.0)  # fill the box
    D1, _ = continuous_maps(seed + 1, (g.n[2], g.n[1], g.n[0]), g.cell, footprint=2.0)
    return (D0 - R0).astype(np.float32), (D1 - R0).astype(np.float32)


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
def test_cross_padded_vs_oracle(torch, precision):
    from paper_2108_00015_gb300 import CkError
    g = GridSpec((26, 22, 18), (0.0, 0.0, 0.0), 10.0, False)
    shells, width = (20.0, 30.0, 40.0), 10.0
    f0, f1 = _two_maps(g, 7)
    ref = O.field_sums(g, shells, width, f0, f1, orders=(2, 3), engine="direct")
    plan = _plan(g, shells, width, 3, precision, padded=True)
    res = plan.compute_cross(dev(torch, f0), dev(torch, f1), orders=(2, 3), out="host")
    _check(res, ref, len(shells), (2, 3))
    # host fields through the staging buffers give the same sums
    hres = plan.compute_cross(f0, f1, orders=(2, 3), out="host")
    for n in (2, 3):
        assert np.array_equal(hres["num"][n].numpy(), res["num"][n].numpy())
    plan.close()
    # maps that fill a box plan (transform lengths 24, 20, 18) reach its
    # faces: the guard band is reported
    gb = GridSpec((24, 20, 18), (0.0, 0.0, 0.0), 10.0, False)
    b0, b1 = _two_maps(gb, 9)
    box = _plan(gb, shells, width, 3, precision, padded=False)
    with pytest.raises(CkError) as e:
        box.compute_cross(dev(torch, b0), dev(torch, b1), orders=(2, 3), out="host")
    assert e.value.code == 6
    box.close()


def test_cross_of_a_field_with_itself(torch):
    """compute_cross(f, f) is compute_continuous of the over-density f."""
    g = GridSpec((24, 24, 24), (0.0, 0.0, 0.0), 10.0, True)
    f, _ = _two_maps(g, 11)
    plan = _plan(g, (20.0, 30.0), 10.0, 3, "fp32")
    a = plan.compute_cross(dev(torch, f), dev(torch, f), orders=(2, 3), out="host")
    b = plan.compute_continuous(dev(torch, f), None, orders=(2, 3), out="host")
    for n in (2, 3):
        assert np.array_equal(a["num"][n].numpy(), b["num"][n].numpy())
    plan.close()


@pytest.mark.parametrize("precision,padded", [("fp32", False), ("split_tf32", False), ("fp32", True)])
def test_product_map(torch, precision, padded):
    from paper_2108_00015_gb300 import CkError
    periodic = not padded
    g = GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, periodic)
    shells, width = (20.0, 35.0, 50.0), 10.0
    data = neyman_scott_box(41, 300, 12, 10.0, 320.0)
    rand = uniform_box(42, 40000, 320.0)
    plan = _plan(g, shells, width, 2, precision, padded=padded)
    with pytest.raises(CkError):
        plan.product_map(0)                                   # no randoms yet
    plan.set_randoms(*dev_cat(torch, rand))
    res = plan.compute(*dev_cat(torch, data), orders=(2,), out="host")
    ref = O.correlate(g, shells, width, data, rand, orders=(2,), engine="fft" if periodic else "direct")
    nb = g.n_cells
    for s in range(len(shells)):
        m = plan.product_map(s, out="host").astype(np.float64)
        den2 = float(ref["den2"][s])
        want = O.product_map(ref["N"], ref["W"][s], den2, nb)
        # scale of each cell's terms: |N| (|N| *** K_s) / <B_0 B_s>
        absw = O.convolve_direct(np.abs(ref["N"]), ref["offsets"][s], periodic)
        scale = np.abs(ref["N"]) * absw / (den2 / nb)
        assert normwise(m, want, scale + 1e-30) <= TOL, s
        # the sum rule: sum_r map <B_0 B_s> = num_2(s) of the same compute
        avg = float(res["den"][2].numpy()[s]) / nb
        assert abs(float(m.sum()) * avg - float(res["num"][2].numpy()[s])) <= TOL * float(ref["abs_num2"][s])
    # device output equals host output
    md = plan.product_map(1).cpu().numpy()
    assert np.array_equal(md, plan.product_map(1, out="host"))
    # after a field compute the map is refused
    f = np.zeros((32, 32, 32), np.float32)
    f[3, 4, 5] = 1.0
    plan.compute_continuous(dev(torch, f), None, orders=(2,), out="host")
    with pytest.raises(CkError) as e:
        plan.product_map(0)
    assert e.value.code == 1
    plan.close()


def test_fields_leave_randoms_intact(torch):
    """A field compute between two catalog computes (host fields, staged
    through plan scratch) leaves the randoms' grid, state and denominators
    as they were: the second catalog compute is bit-identical to the first."""
    g = GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, True)
    shells = (20.0, 35.0)
    data = neyman_scott_box(51, 300, 12, 10.0, 320.0)
    rand = uniform_box(52, 40000, 320.0)
    for precision in ("fp32", "split_tf32"):
        plan = _plan(g, shells, 10.0, 3, precision)
        plan.set_randoms(*dev_cat(torch, rand))
        first = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
        D, R = continuous_maps(53, (32, 32, 32), g.cell)
        plan.compute_continuous(D, R, orders=(2, 3), out="host")                 # host maps
        plan.compute_cross(D, R, orders=(2,), out="host")
        again = plan.compute(*dev_cat(torch, data), orders=(2, 3), out="host")
        for n in (2, 3):
            for key in ("xi", "num", "den"):
                assert np.array_equal(first[key][n].numpy(), again[key][n].numpy()), (precision, n, key)
        plan.close()


def test_degenerate_fields(torch):
    """An all-zero map, D = R (delta = 0) and R = 0 everywhere (no survey)
    give sums of exactly 0.  A single nonzero cell has no pair in any shell
    (the shells exclude the zero offset): its sums vanish to the transform's
    rounding, against the size of its products (2^n |O_s|)."""
    g = GridSpec((24, 24, 24), (0.0, 0.0, 0.0), 10.0, True)
    plan = _plan(g, (20.0, 30.0), 10.0, 3, "fp32")
    zero = np.zeros((24, 24, 24), np.float32)
    R = np.full((24, 24, 24), 1.5, np.float32)
    one = zero.copy()
    one[5, 6, 7] = 2.0
    for d, r in ((zero, None), (R, R), (R, zero)):
        res = plan.compute_continuous(dev(torch, d), None if r is None else dev(torch, r), orders=(2, 3),
                                      out="host")
        for n in (2, 3):
            assert float(np.abs(res["num"][n].numpy()).max()) == 0.0
    res = plan.compute_continuous(dev(torch, one), None, orders=(2, 3), out="host")
    big = max(plan.shell_size)
    for n in (2, 3):
        assert float(np.abs(res["num"][n].numpy()).max()) <= 1e-5 * 2.0 ** n * big ** (n - 1)
    plan.close()
