"""ck_contract_static, the contraction entry point that allocates nothing:
its scratch is a fixed device array inside the library, so callers that
cannot allocate device memory (a foreign memory pool, an allocation-free
region) can still run the summation.  Checked through the C ABI against
ck_contract (which uses plan workspace) on two calls in a row.  Kept in a
file collected last, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec
from tests.gpu_util import cuda_torch, dev, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("ns,orders", [(16, (2, 3)), (5, (2, 3, 4, 5)), (3, (3,))])
def test_static_contraction_matches_plan_contraction(ns, orders):
    torch = cuda_torch()
    from paper_2108_00015_gb300 import conker
    g = GridSpec((40, 24, 30), (0.0, 0.0, 0.0), 1.0, True)
    nc = g.n_cells
    rng = np.random.default_rng(100 + ns)
    w0 = rng.normal(size=nc).astype(np.float32)
    bank = rng.normal(size=(ns, nc)).astype(np.float32)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((ns, stride), np.float32)
    B[:, :nc] = bank
    w = dict(grid=g, shells=tuple(1.0 + 0.05 * i for i in range(ns)), width=1.0)
    plan = plan_for(w, max_order=max(orders))
    tw0, tB = dev(torch, w0), dev(torch, B)
    want = plan.contract(tw0, tB, stride, orders=orders)
    for call in range(2):  # the shared scratch keeps the previous call's contents
        got = conker.contract_static(tw0, tB, stride, nc, ns, orders=orders)
        torch.cuda.synchronize()
        for n in orders:
            ref, aref = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
            a = got[n].cpu().numpy()
            assert normwise(a, want[n].cpu().numpy(), aref) <= TOL, f"call {call} order {n}"
            assert normwise(a, ref, aref) <= TOL, f"call {call} order {n} vs oracle"
    plan.close()


def test_static_contraction_limits():
    torch = cuda_torch()
    from paper_2108_00015_gb300 import CkError, conker
    x = torch.zeros(1024, dtype=torch.float32, device="cuda")
    with pytest.raises(CkError) as e:
        conker.contract_static(x, x, 64, 64, 17, orders=(2, 3))
    assert e.value.code == 10  # beyond the fixed scratch
    with pytest.raises(CkError) as e:
        conker.contract_static(x, x, 64, 64, 6, orders=(4,))
    assert e.value.code == 10
    with pytest.raises(CkError) as e:
        conker.contract_static(x, x, 63, 64, 4, orders=(2,))
    assert e.value.code == 1
