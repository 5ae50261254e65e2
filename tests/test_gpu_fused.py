"""The mixed-precision form (CK_PREC_SPLIT_TF32): the fused convolution +
summation pass (inverse x transform and the order-2/3 product sums of Eq. 11
on the tensor cores in one kernel, no bank in global memory) against the FP64
oracle, for every padded shell count (2, 4, 8, 16), an
odd half-length x axis (runtime transform length) and against the plan's
unfused path on the same catalog."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _box(n, cell, shells, width, seed):
    g = GridSpec(n, (0.0, 0.0, 0.0), cell, True)
    L = np.array(n, np.float64) * cell
    data = neyman_scott_box(seed, 300, 12, 1.5 * cell, float(L.min()))
    rand = uniform_box(seed + 1, 60 * int(np.prod(n)) // 64, float(L.min()))
    # keep the catalogs inside the (possibly non-cubic) box
    def clip(c):
        from synth import Catalog
        sel = (c.x < L[0]) & (c.y < L[1]) & (c.z < L[2])
        return Catalog(c.x[sel], c.y[sel], c.z[sel])
    return dict(grid=g, shells=tuple(shells), width=width, data=clip(data), randoms=clip(rand))


def _run(torch, w, max_order=3, precision="split_tf32"):
    plan = plan_for(w, max_order=max_order, precision=precision)
    plan.set_randoms(*dev_cat(torch, w["randoms"]))
    res = plan.compute(*dev_cat(torch, w["data"]), orders=(2, 3), out="host")
    return plan, res


def _check(res, ref, ns):
    for n in (2, 3):
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
            e = normwise(got, want, scale)
            assert e <= TOL, f"order {n} {key}: normwise error {e:.3e}"


def test_fused_selection(torch):
    w = _box((32, 32, 32), 10.0, (20.0, 40.0), 10.0, 1)
    for mo, prec, want in ((2, "split_tf32", True), (3, "split_tf32", True), (3, "fp32", False),
                           (4, "fp32", False), (3, "fp64", False)):
        p = plan_for(w, max_order=mo, precision=prec)
        assert p.fused is want, (mo, prec)
        p.close()
    p = plan_for(w, max_order=4, precision="split_tf32")  # bank + tensor-core blocked product
    assert not p.fused
    p.close()
    w17 = _box((32, 32, 32), 10.0, tuple(20.0 + 5 * i for i in range(17)), 5.0, 1)
    p = plan_for(w17, max_order=3, precision="split_tf32")
    assert not p.fused
    p.close()


@pytest.mark.parametrize("ns", [1, 3, 5, 8, 9, 16])
def test_fused_shell_counts(torch, ns):
    shells = tuple(20.0 + 7.5 * i for i in range(ns))
    w = _box((32, 32, 32), 10.0, shells, 7.5, 10 + ns)
    ref = O.correlate(w["grid"], shells, w["width"], w["data"], w["randoms"], orders=(2, 3), engine="fft")
    plan, res = _run(torch, w)
    assert plan.fused
    _check(res, ref, ns)
    plan.close()


def test_fused_odd_half_length(torch):
    """x axis of 30 cells: half-length 15 (odd), runtime transform length and
    staged rows of odd length, in both the fused and the unfused path."""
    shells = (20.0, 35.0, 50.0)
    w = _box((30, 32, 20), 10.0, shells, 10.0, 31)
    ref = O.correlate(w["grid"], shells, w["width"], w["data"], w["randoms"], orders=(2, 3), engine="fft")
    for prec in ("split_tf32", "fp32"):
        plan, res = _run(torch, w, precision=prec)
        assert plan.fused is (prec == "split_tf32")
        _check(res, ref, len(shells))
        for s in range(len(shells)):
            got = plan.bank(s).cpu().numpy()
            want = ref["W"][s]
            assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), f"shell {s}"
        plan.close()


def test_fused_vs_unfused(torch):
    """Same catalog, 12 shells on a 64^3 box: the mixed plan (fused pass) and
    the plain FP32 one (bank + register contraction) agree with the oracle on
    the order-2/3 sums, and the mixed plan's recomputed bank equals the stored
    one."""
    shells = tuple(15.0 + 6.0 * i for i in range(12))
    w = _box((64, 64, 64), 5.0, shells, 6.0, 41)
    ref = O.correlate(w["grid"], shells, w["width"], w["data"], w["randoms"], orders=(2, 3), engine="fft")
    pf, rf = _run(torch, w, precision="split_tf32")
    pu, ru = _run(torch, w, precision="fp32")
    assert pf.fused and not pu.fused
    _check(rf, ref, 12)
    _check(ru, ref, 12)
    for s in (0, 5, 11):
        a = pf.bank(s).cpu().numpy()
        b = pu.bank(s).cpu().numpy()
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()
    pf.close()
    pu.close()


def test_fused_x512_every_order3_entry(torch):
    """The survey step's fused kernel as it runs there: a 512-cell x axis
    (half-length M = 256, the 16 x 16 register transform) with 16 shells
    (no padded lines).  A periodic 512 x 24 x 20 box of unit cells keeps the
    oracle fast; every order-2 and order-3 entry of num and den is compared,
    normwise, with the oracle's FFT engine (itself pinned to the direct
    convolution)."""
    n = (512, 24, 20)
    L = tuple(float(v) for v in n)
    shells = tuple(1.0 + 0.45 * i for i in range(16))
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, True)
    w = dict(grid=g, shells=shells, width=0.5, data=neyman_scott_box(71, 700, 10, 1.5, L),
             randoms=uniform_box(72, 250_000, L))
    ref = O.correlate(g, shells, w["width"], w["data"], w["randoms"], orders=(2, 3), engine="fft")
    plan, res = _run(torch, w)
    assert plan.fused
    _check(res, ref, len(shells))
    # and the same sums from the plain FP32 path on the same catalog
    pu, ru = _run(torch, w, precision="fp32")
    _check(ru, ref, len(shells))
    pu.close()
    plan.close()
