"""The failure path of the bounded device waits, made to run out on purpose
without faulting or hanging anything: ck_debug_force_timeout makes each
consumer warp of the register contraction wait, with a 50 us limit, on an
mbarrier that nothing arrives at, so every launch gives up, records
CK_ERR_TIMEOUT, waits (with the default limit) for the bulk copies it has
issued and returns.  The plan's
status word then reports the timeout and the allocation-free entry point
returns NaN; with the default limit restored, the same calls give finite
sums equal to the oracle's."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec
from tests.gpu_util import cuda_torch, dev, normwise, plan_for

pytestmark = pytest.mark.gpu


def _inputs(ns, nc, seed):
    rng = np.random.default_rng(seed)
    w0 = rng.normal(size=nc).astype(np.float32)
    bank = rng.normal(size=(ns, nc)).astype(np.float32)
    stride = (nc + 63) // 64 * 64
    B = np.zeros((ns, stride), np.float32)
    B[:, :nc] = bank
    return w0, bank, B, stride


def test_consumer_timeout_reported_and_recovered():
    torch = cuda_torch()
    from paper_2108_00015_gb300 import conker
    g = GridSpec((64, 48, 40), (0.0, 0.0, 0.0), 1.0, True)
    nc = g.n_cells
    ns = 6
    w0, bank, B, stride = _inputs(ns, nc, 5)
    w = dict(grid=g, shells=tuple(1.0 + 0.3 * i for i in range(ns)), width=1.0)
    plan = plan_for(w, max_order=3)  # plain FP32: the register contraction
    tw0, tB = dev(torch, w0), dev(torch, B)
    assert plan.status() == 0
    try:
        conker.force_timeout(50_000)
        got = plan.contract(tw0, tB, stride, orders=(2, 3))
        torch.cuda.synchronize()
        assert plan.status() == 8  # CK_ERR_TIMEOUT, read (and cleared) from the status word
        st = conker.contract_static(tw0, tB, stride, nc, ns, orders=(2, 3))
        torch.cuda.synchronize()
        for n in (2, 3):
            assert torch.isnan(st[n]).all(), f"order {n}: a timed-out static call returns NaN"
        del got
    finally:
        conker.force_timeout(0)
    # the context stays usable and the default limit is back
    want = plan.contract(tw0, tB, stride, orders=(2, 3))
    st = conker.contract_static(tw0, tB, stride, nc, ns, orders=(2, 3))
    torch.cuda.synchronize()
    assert plan.status() == 0
    for n in (2, 3):
        ref, aref = O.product_sums(w0.astype(np.float64), [b.astype(np.float64) for b in bank], n)
        assert normwise(want[n].cpu().numpy(), ref, aref) <= 1e-5
        assert normwise(st[n].cpu().numpy(), ref, aref) <= 1e-5
    plan.close()
