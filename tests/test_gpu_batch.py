"""The batched form (ck_batch_compute): catalogs over several grid classes,
each class's compute sequence replayed from a captured CUDA graph, against
per-catalog ck_compute on the same plans (bit for bit) and the FP64 oracle."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec, neyman_scott_box, uniform_box
from paper_2108_00015_gb300 import batch_compute
from tests.gpu_util import cuda_torch, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

SHELLS = (20.0, 30.0, 45.0)


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _class(n, cell, seed):
    g = GridSpec((n, n, n), (0.0, 0.0, 0.0), cell, True)
    return dict(grid=g, shells=SHELLS, width=10.0, randoms=uniform_box(seed, 40 * n ** 3 // 64, n * cell))


def _mocks(classes):
    out = []
    for i, (j, n_par, sigma) in enumerate([(0, 60, 6.0), (1, 120, 9.0), (0, 200, 12.0), (1, 30, 4.0), (0, 90, 8.0)]):
        g = classes[j]["grid"]
        out.append((j, neyman_scott_box(100 + i, n_par, 20, sigma, g.length[0])))
    return out


@pytest.mark.parametrize("precision,max_order", [("split_tf32", 3), ("fp32", 3), ("split_tf32", 4)])
def test_batch_matches_compute(torch, precision, max_order):
    classes = [_class(32, 10.0, 7), _class(40, 8.0, 8)]
    plans = []
    for c in classes:
        p = plan_for(c, max_order=max_order, precision=precision)
        p.set_randoms(*dev_cat(torch, c["randoms"]))
        plans.append(p)
    mocks = _mocks(classes)
    orders = tuple(range(2, max_order + 1))
    cats = [(*dev_cat(torch, m), j) for j, m in mocks]
    res = batch_compute(plans, cats, orders=orders, out="host")
    for (j, m), r in zip(mocks, res):
        single = plans[j].compute(*dev_cat(torch, m), orders=orders, out="host")
        for n in orders:
            for key in ("xi", "num", "den"):
                assert np.array_equal(r[key][n].numpy(), single[key][n].numpy()), (j, n, key)
    # one catalog of each class against the oracle
    for (j, m), r in list(zip(mocks, res))[:2]:
        c = classes[j]
        ref = O.correlate(c["grid"], SHELLS, c["width"], m, c["randoms"], orders=orders, engine="fft")
        for n in orders:
            want = O.dense_tensor(ref[f"num{n}"], len(SHELLS), n - 1)
            scale = O.dense_tensor(ref[f"abs_num{n}"], len(SHELLS), n - 1)
            assert normwise(r["num"][n].numpy(), want, scale) <= 1e-5
    for p in plans:
        p.close()


def test_batch_errors(torch):
    from paper_2108_00015_gb300.conker import CkError
    c = _class(32, 10.0, 9)
    p = plan_for(c, max_order=3, precision="split_tf32")
    m = neyman_scott_box(5, 50, 20, 8.0, 320.0)
    with pytest.raises(CkError):  # randoms not set
        batch_compute([p], [(*dev_cat(torch, m), 0)])
    p.set_randoms(*dev_cat(torch, c["randoms"]))
    with pytest.raises(CkError):  # host positions
        batch_compute([p], [(m.x, m.y, m.z, 0)])
    with pytest.raises(CkError):  # plan index out of range
        batch_compute([p], [(*dev_cat(torch, m), 1)])
    p.close()


def test_batch_with_thin_tiles_beside_tensor_cores(torch):
    """16 shells, orders 2..4: one tensor-core tile and a thin tile, the thin
    tile on the plan's second stream inside the captured graph; the batched
    results equal ck_compute's bit for bit with the overlap on and off."""
    shells = tuple(20.0 + 5.0 * i for i in range(16))
    classes = [dict(c, shells=shells, width=5.0) for c in (_class(32, 10.0, 17), _class(40, 8.0, 18))]
    mocks = _mocks(classes)
    for overlap in (1, 0):
        plans = []
        for c in classes:
            p = plan_for(c, max_order=4, precision="split_tf32")
            p.set_tuning(8, 8, 8, 2, 32, overlap)
            p.set_randoms(*dev_cat(torch, c["randoms"]))
            plans.append(p)
        cats = [(*dev_cat(torch, m), j) for j, m in mocks]
        res = batch_compute(plans, cats, orders=(2, 3, 4), out="host")
        for (j, m), r in zip(mocks, res):
            single = plans[j].compute(*dev_cat(torch, m), orders=(2, 3, 4), out="host")
            for n in (2, 3, 4):
                for key in ("xi", "num", "den"):
                    assert np.array_equal(r[key][n].numpy(), single[key][n].numpy()), (overlap, j, n, key)
        for p in plans:
            p.close()
