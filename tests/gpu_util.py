"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def cuda_torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__ as g
    g.build()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_cat(torch, c):
    return dev(torch, c.x), dev(torch, c.y), dev(torch, c.z)


def normwise(got, want, scale):
    """max |got - want| / scale, elementwise scale (sum of |terms|)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.asarray(scale, np.float64)
    return float(np.max(np.abs(got - want) / np.maximum(scale, 1e-300)))


def plan_for(w, max_order=3, precision="fp32", rule="center_bin"):
    from paper_2108_00015_gb300 import Plan
    g = w["grid"]
    return Plan(g.n, g.origin, g.cell, g.periodic, w["shells"], w["width"], max_order=max_order,
                precision=precision, rule=rule)
