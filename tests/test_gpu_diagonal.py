"""The equidistant n-point functions alone (ck_compute_diagonal, Eq. 14):
xi_n(s, .., s) = sum W0 W_s^(n-1) / sum B0 B_s^(n-1) for every shell, against
the FP64 oracle's xi_diagonal on the oracle's own fields, for the fused
mixed plan (no bank: diagonal entries of the order-2/3 sums), the mixed plan
that keeps the bank and the plain FP32 plan (one pass over the bank, orders
2..5), a grid whose cell count is not a multiple of the kernel's 16-byte
loads (ragged tail), and against the diagonal of ck_compute's full tensor."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, neyman_scott_box, uniform_box
from tests.gpu_util import cuda_torch, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _box(n, cell, shells, width, seed):
    g = GridSpec(n, (0.0, 0.0, 0.0), cell, True)
    L = np.array(n, np.float64) * cell
    data = neyman_scott_box(seed, 200, 12, 1.5 * cell, float(L.min()))
    rand = uniform_box(seed + 1, 50 * int(np.prod(n)) // 64, float(L.min()))

    def clip(c):
        sel = (c.x < L[0]) & (c.y < L[1]) & (c.z < L[2])
        return Catalog(c.x[sel], c.y[sel], c.z[sel])
    return dict(grid=g, shells=tuple(shells), width=width, data=clip(data), randoms=clip(rand))


def _oracle(w, orders):
    ref = O.correlate(w["grid"], w["shells"], w["width"], w["data"], w["randoms"], orders=(2,), engine="fft")
    out = {}
    for n in orders:
        xi, num, den, anum, aden = [], [], [], [], []
        for s in range(len(w["shells"])):
            Ws, Bs = ref["W"][s], ref["B"][s]
            num.append(float(np.sum(ref["N"] * Ws ** (n - 1))))
            den.append(float(np.sum(ref["Rt"] * Bs ** (n - 1))))
            anum.append(float(np.sum(np.abs(ref["N"] * Ws ** (n - 1)))))
            aden.append(float(np.sum(np.abs(ref["Rt"] * Bs ** (n - 1)))))
            xi.append(O.xi_diagonal(ref["N"], Ws, ref["Rt"], Bs, n))
        out[n] = dict(xi=np.array(xi), num=np.array(num), den=np.array(den), anum=np.array(anum),
                      aden=np.array(aden))
    return out


def _run(torch, w, orders, max_order, precision, diag_randoms=False):
    plan = plan_for(w, max_order=max_order, precision=precision)
    if diag_randoms:
        plan.set_randoms_diagonal(*dev_cat(torch, w["randoms"]))
    else:
        plan.set_randoms(*dev_cat(torch, w["randoms"]))
    res = plan.compute_diagonal(*dev_cat(torch, w["data"]), orders=orders, out="host")
    return plan, res


def _check(res, ref, orders):
    for n in orders:
        e = normwise(res["num"][n].numpy(), ref[n]["num"], ref[n]["anum"])
        assert e <= TOL, f"order {n} num: {e:.3e}"
        e = normwise(res["den"][n].numpy(), ref[n]["den"], ref[n]["aden"])
        assert e <= TOL, f"order {n} den: {e:.3e}"
        got, want = res["xi"][n].numpy(), ref[n]["xi"]
        # xi = num / den: the num error relative to |den| bounds the xi error
        scale = ref[n]["anum"] / np.abs(ref[n]["den"])
        assert np.max(np.abs(got - want) / scale) <= 4 * TOL, f"order {n} xi"


@pytest.mark.parametrize("diag_randoms", [False, True])
@pytest.mark.parametrize("precision,max_order,orders", [
    ("split_tf32", 3, (2, 3)),       # fused pass: no bank
    ("split_tf32", 5, (2, 3, 4, 5)),  # bank kept, tensor-core plan
    ("fp32", 5, (2, 3, 4, 5)),
    ("fp32", 4, (3, 4)),
])
def test_diagonal_vs_oracle(torch, precision, max_order, orders, diag_randoms):
    """Denominators from ck_set_randoms (every multiset) or from
    ck_set_randoms_diagonal (the (s, .., s) ones alone)."""
    shells = (20.0, 30.0, 40.0, 55.0)
    w = _box((32, 32, 32), 10.0, shells, 10.0, 7)
    ref = _oracle(w, orders)
    plan, res = _run(torch, w, orders, max_order, precision, diag_randoms)
    assert plan.fused is (precision == "split_tf32" and max_order <= 3)
    _check(res, ref, orders)
    plan.close()


def test_diagonal_ragged_cells(torch):
    """30 x 18 x 10 cells (5400: 16-byte groups plus a partial CTA range),
    4 shells inside half the shortest periodic axis."""
    shells = (1.5, 2.25, 3.0, 3.75)
    w = _box((30, 18, 10), 1.0, shells, 0.75, 11)
    ref = _oracle(w, (2, 3, 4, 5))
    plan, res = _run(torch, w, (2, 3, 4, 5), 5, "fp32", diag_randoms=True)
    _check(res, ref, (2, 3, 4, 5))
    plan.close()


def test_diagonal_randoms_state(torch):
    """After ck_set_randoms_diagonal a plan that keeps the bank has only the
    diagonal denominators: ck_compute refuses (CK_ERR_NO_RANDOMS, 11) until
    ck_set_randoms; a fused plan sums every multiset and computes as usual."""
    from paper_2108_00015_gb300.conker import CkError
    w = _box((32, 32, 32), 10.0, (20.0, 30.0), 10.0, 5)
    d = dev_cat(torch, w["data"])
    plan = plan_for(w, max_order=4, precision="fp32")
    plan.set_randoms_diagonal(*dev_cat(torch, w["randoms"]))
    with pytest.raises(CkError) as e:
        plan.compute(*d, orders=(2, 3))
    assert e.value.code == 11
    plan.set_randoms(*dev_cat(torch, w["randoms"]))
    plan.compute(*d, orders=(2, 3))
    plan.close()
    fused = plan_for(w, max_order=3, precision="split_tf32")
    fused.set_randoms_diagonal(*dev_cat(torch, w["randoms"]))
    assert fused.compute(*d, orders=(2, 3))["status"] in (0, 7)
    fused.close()


def test_diagonal_matches_full_tensor(torch):
    """The diagonal mode's entries equal the diagonal of ck_compute's dense
    tensors (to rounding of the summation order) on the same catalog."""
    shells = tuple(15.0 + 6.0 * i for i in range(8))
    w = _box((32, 32, 32), 5.0, shells, 6.0, 21)
    for precision, mo in (("split_tf32", 3), ("split_tf32", 4), ("fp32", 5)):
        orders = tuple(range(2, mo + 1))
        plan = plan_for(w, max_order=mo, precision=precision)
        plan.set_randoms(*dev_cat(torch, w["randoms"]))
        d = dev_cat(torch, w["data"])
        full = plan.compute(*d, orders=orders, out="host")
        diag = plan.compute_diagonal(*d, orders=orders, out="host")
        for n in orders:
            T = full["num"][n].numpy()
            want = np.array([T[(s,) * (n - 1)] for s in range(len(shells))])
            got = diag["num"][n].numpy()
            assert np.allclose(got, want, rtol=2e-5, atol=1e-6 * np.abs(want).max()), (precision, n)
            Td = full["den"][n].numpy()
            dwant = np.array([Td[(s,) * (n - 1)] for s in range(len(shells))])
            assert np.array_equal(diag["den"][n].numpy(), dwant), (precision, n)
        assert np.array_equal(diag["dropped"].numpy(), full["dropped"].numpy())
        plan.close()
