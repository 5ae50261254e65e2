"""The autotuner's choices change launch shapes only.  Every choice of tile
width of the 512-point strided passes (forward, K^ z pass, inverse y pass)
gives transforms, and so sums, identical bit for bit to the defaults', and
every choice of contraction CTAs per SM gives sums within the gate of the
oracle's; ck_plan_autotune keeps one of the candidates and the results stay
the same."""
import itertools

import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu


def _case():
    n = (32, 512, 512)
    L = tuple(float(v) for v in n)
    g = GridSpec(n, (0.0, 0.0, 0.0), 1.0, True)
    return dict(grid=g, shells=(1.5, 2.5, 3.5), width=1.0, data=neyman_scott_box(61, 800, 10, 1.5, L),
                randoms=uniform_box(62, 400_000, L))


@pytest.mark.parametrize("precision", ["split_tf32", "fp32"])
def test_tile_widths_bit_identical(precision):
    torch = cuda_torch()
    w = _case()
    plan = plan_for(w, max_order=3, precision=precision)
    d, r = dev_cat(torch, w["data"]), dev_cat(torch, w["randoms"])

    def run():
        plan.set_randoms(*r)
        res = plan.compute(*d, orders=(2, 3), out="host")
        return {k: res[k][n].numpy().copy() for k in ("num", "den") for n in (2, 3)}, res["status"]

    base, st = run()
    assert st == 0
    assert plan.tuning()["tuned"] is False
    for fwd, zreg, yinv in itertools.product((8, 16), repeat=3):
        plan.set_tuning(fwd, zreg, yinv, 2)
        got, st = run()
        assert st == 0
        for k in base:
            assert np.array_equal(got[k], base[k]), (fwd, zreg, yinv, k)
    plan.set_tuning()
    plan.set_randoms(*r)
    t = plan.autotune()
    assert t["tuned"] and t["fwd_cols"] in (8, 16) and t["zreg_cols"] in (8, 16) and t["yinv_cols"] in (8, 16)
    got, st = run()
    for k in base:
        assert np.array_equal(got[k], base[k]), k
    # after a compute the catalog's field is the one timed
    plan.autotune()
    got, st = run()
    assert st == 0
    for k in base:
        assert np.array_equal(got[k], base[k]), k
    plan.close()


@pytest.mark.parametrize("precision", ["split_tf32", "split_bf16"])
def test_contraction_ctas_per_sm(precision):
    torch = cuda_torch()
    g = GridSpec((24, 20, 18), (0.0, 0.0, 0.0), 1.0, True)
    rng = np.random.default_rng(63)
    nc, ns = g.n_cells, 8
    w0 = rng.normal(size=nc).astype(np.float32)
    bank = rng.normal(size=(ns, nc)).astype(np.float32)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((ns, stride), np.float32)
    B[:, :nc] = bank
    w = dict(grid=g, shells=tuple(1.0 + 0.05 * i for i in range(ns)), width=1.0)
    plan = plan_for(w, max_order=5, precision=precision)
    tol = 1e-5 if precision == "split_tf32" else 5e-5
    for k in (1, 2, 3):
        plan.set_tuning(8, 8, 8, k)
        sums = plan.contract(dev(torch, w0), dev(torch, B), stride, orders=(2, 3, 4, 5))
        for n in (2, 3, 4, 5):
            want, awant = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
            assert normwise(sums[n].cpu().numpy(), want, awant) <= tol, (k, n)
    plan.close()
