"""Multi-rank use of the library: one catalog (or one sky region) per rank,
or one catalog cut into slabs along z.

ConKer's numerators and denominators are sums over cells, so independent
regions combine by adding them before the division (Eq. 19 combines the two
galactic caps that way).  Ranks therefore need no data exchange while they
run the path; the only collective is one FP64 sum of the num and den tensors
when regions of one survey were spread over ranks.

A single catalog too large for one device splits into slabs of z planes:
each rank grids its owned planes plus a halo of max|m_z| planes on either
side (the kernels' reach, clipped at the catalog's faces) into a zero-padded
box of its own, sums over its owned planes only (ck_plan_set_region) with
the alpha of the whole catalog (one all-reduce of the owned point counts),
and the slabs' num and den add up to the undivided catalog's.
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np


def shard(n_units: int, rank: int, world: int) -> Sequence[int]:
    """The units (catalogs, mocks, regions) rank `rank` of `world` owns:
    a contiguous block, sizes differing by at most one."""
    base, extra = divmod(int(n_units), int(world))
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def combine_regions(num: Dict[int, "object"], den: Dict[int, "object"], group=None
                    ) -> Tuple[Dict[int, "object"], Dict[int, "object"], Dict[int, "object"]]:
    """Sum every rank's num and den tensors (FP64) and return
    (num, den, xi) of the union, xi = num / den with NaN where den <= 0."""
    import torch
    import torch.distributed as dist
    out_num, out_den, out_xi = {}, {}, {}
    for n in sorted(num):
        a = num[n].to(torch.float64).clone()
        b = den[n].to(torch.float64).clone()
        if dist.is_available() and dist.is_initialized():
            dist.all_reduce(a, op=dist.ReduceOp.SUM, group=group)
            dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
        xi = torch.where(b > 0, a / torch.where(b > 0, b, torch.ones_like(b)), torch.full_like(b, float("nan")))
        out_num[n], out_den[n], out_xi[n] = a, b, xi
    return out_num, out_den, out_xi


def slab_planes(nz: int, parts: int, rank: int) -> Tuple[int, int]:
    """Owned planes [z0, z1) of slab `rank` of `parts` (contiguous, sizes
    differing by at most one)."""
    r = shard(nz, rank, parts)
    return r.start, r.stop


def slab_box(nz: int, z0: int, z1: int, halo: int) -> Tuple[int, int]:
    """Planes [lo, hi) of the slab's box: the owned planes and a halo of
    `halo` planes on either side, clipped to the catalog's [0, nz)."""
    return max(0, z0 - halo), min(nz, z1 + halo)


def in_planes(z, origin_z: float, cell: float, lo: int, hi: int) -> np.ndarray:
    """Points whose z cell lies in [lo, hi): edge_lo <= z < edge_hi with the
    cell edges origin + k cell in FP64, compared with the float32
    coordinates exactly as the gridding does; a slab box whose origin is the
    catalog's shifted by lo cells assigns the same cells when those edges are
    exact (a dyadic origin and cell, for instance)."""
    zd = np.asarray(z, np.float32).astype(np.float64)
    e_lo = np.float64(origin_z) + np.float64(lo) * np.float64(cell)
    e_hi = np.float64(origin_z) + np.float64(hi) * np.float64(cell)
    return (zd >= e_lo) & (zd < e_hi)


def global_alpha(n_data_owned: float, n_rand_owned: float, group=None) -> float:
    """alpha of the whole catalog from every rank's owned-plane totals (one
    FP64 all-reduce): sum D / sum R over all slabs."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(n_data_owned), float(n_rand_owned)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t[0] / t[1]) if t[1] > 0 else 0.0
