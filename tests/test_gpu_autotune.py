"""The autotuner's choices.  Under either z route (the shells' short
filters or the forward and K^ z passes), every choice of tile width of the
512-point strided passes (forward, K^ z pass, inverse y pass) gives
transforms, and so sums, identical bit for bit to that route's defaults;
the two routes' sums agree with the oracle's within the gate; every choice
of contraction CTAs per SM gives sums within the gate of the oracle's; and
ck_plan_autotune keeps one of the candidates, whose results are the chosen
route's."""
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
        return {f"{k}{n}": res[k][n].numpy().copy() for k in ("num", "den") for n in (2, 3)}, res["status"]

    assert plan.tuning()["tuned"] is False
    assert plan.tuning()["z_direct"] == 1  # 3.5-cell shells: short filters
    bases = {}
    for zd in (0, 1):
        plan.set_tuning(z_direct=zd)
        bases[zd], st = run()
        assert st == 0
        for fwd, zreg, yinv in itertools.product((8, 16), repeat=3):
            plan.set_tuning(fwd, zreg, yinv, 2, z_direct=zd)
            got, st = run()
            assert st == 0
            for k in bases[zd]:
                assert np.array_equal(got[k], bases[zd][k]), (zd, fwd, zreg, yinv, k)
    # the routes sum in different orders: both within the oracle's gate
    ref = O.correlate(w["grid"], w["shells"], w["width"], w["data"], w["randoms"], orders=(2, 3), engine="fft")
    ns = len(w["shells"])
    for zd in (0, 1):
        for n in (2, 3):
            for key, akey in (("num", "abs_num"), ("den", "abs_den")):
                want = O.dense_tensor(ref[f"{key}{n}"], ns, n - 1)
                scale = O.dense_tensor(ref[f"{akey}{n}"], ns, n - 1)
                assert normwise(bases[zd][f"{key}{n}"], want, scale) <= 1e-5, (zd, key, n)
    plan.set_tuning()
    plan.set_randoms(*r)
    t = plan.autotune()
    assert t["tuned"] and t["fwd_cols"] in (8, 16) and t["zreg_cols"] in (8, 16) and t["yinv_cols"] in (8, 16)
    base = bases[t["z_direct"]]
    got, st = run()
    for k in base:
        assert np.array_equal(got[k], base[k]), k
    # after a compute the catalog's field is the one timed
    t = plan.autotune()
    base = bases[t["z_direct"]]
    got, st = run()
    assert st == 0
    for k in base:
        assert np.array_equal(got[k], base[k]), k
    plan.close()


@pytest.mark.parametrize("precision", ["split_tf32", "split_bf16", "split_fp16"])
@pytest.mark.parametrize("ns,orders", [(8, (2, 3, 4, 5)), (8, (2, 3, 4)), (32, (2, 3, 4))])
def test_contraction_tile_choices(precision, ns, orders):
    """Every contraction CTA count and stacked-tile width gives sums within
    the form's gate of the oracle's: stacked tiles (B's hi and lo side by
    side, two MMAs per k-step) cover the order-4 column lists of 8 and 32
    shells (8 and 32 live columns) and, at width 64, the 44-column tile of
    orders up to 5."""
    torch = cuda_torch()
    g = GridSpec((24, 20, 18), (0.0, 0.0, 0.0), 1.0, True)
    rng = np.random.default_rng(63 + ns)
    nc = g.n_cells
    w0 = rng.normal(size=nc).astype(np.float32)
    bank = rng.normal(size=(ns, nc)).astype(np.float32)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((ns, stride), np.float32)
    B[:, :nc] = bank
    w = dict(grid=g, shells=tuple(1.0 + 0.05 * i for i in range(ns)), width=1.0)
    plan = plan_for(w, max_order=max(orders), precision=precision)
    tol = 5e-5 if precision == "split_bf16" else 1e-5
    want = {n: O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n) for n in orders}
    for stack in (0, 32, 64):
        for k in (1, 2, 3):
            for overlap in (0, 1):
                plan.set_tuning(8, 8, 8, k, stack, overlap)
                sums = plan.contract(dev(torch, w0), dev(torch, B), stride, orders=orders)
                for n in orders:
                    assert normwise(sums[n].cpu().numpy(), *want[n]) <= tol, (stack, k, overlap, n)
    plan.close()
