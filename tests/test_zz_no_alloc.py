"""ck_contract_static, the contraction entry point that allocates nothing:
its scratch is a fixed device array inside the library, so callers that
cannot allocate device memory (a foreign memory pool, an allocation-free
region) can still run the summation.  Checked through the C ABI against
ck_contract (which uses plan workspace) on two calls in a row.  Kept in a
file collected last, so that a run stopping at the first failure has
already run every other test."""
import ctypes
import gc

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
    # outputs allocated up front, so that the calls below allocate nothing at all
    got = {n: torch.full_like(want[n], float("nan")) for n in orders}
    arr = (ctypes.c_void_p * (conker.CK_MAX_ORDER + 1))()
    for n, t in got.items():
        arr[n] = t.data_ptr()
    lib = conker.load()
    torch.cuda.synchronize()
    for call in range(2):  # the shared scratch keeps the previous call's contents
        if call == 1:
            gc.collect()  # tensors of earlier tests may still be waiting to be freed
            torch.cuda.synchronize()
            free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        code = lib.ck_contract_static(tw0.data_ptr(), tB.data_ptr(), stride, nc, ns, conker.order_mask(orders),
                                      arr, None)
        assert code == 0
        torch.cuda.synchronize()
        if call == 1:
            # the second call takes no device memory: neither the device's free
            # bytes nor the caching allocator's holdings go down
            assert torch.cuda.mem_get_info()[0] >= free0
            assert torch.cuda.memory_allocated() <= alloc0
        for n in orders:
            ref, aref = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
            a = got[n].cpu().numpy()
            # the same register kernel, CTA count and fixed-order reduction as
            # the plan's contraction: the sums are identical bit for bit
            assert torch.equal(got[n], want[n]), f"call {call} order {n}"
            assert normwise(a, ref, aref) <= TOL, f"call {call} order {n} vs oracle"
            got[n].fill_(float("nan"))
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
