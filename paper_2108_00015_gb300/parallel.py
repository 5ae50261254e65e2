"""Multi-rank use of the library: one catalog (or one sky region) per rank.

ConKer's numerators and denominators are sums over cells, so independent
regions combine by adding them before the division (Eq. 19 combines the two
galactic caps that way).  Ranks therefore need no data exchange while they
run the path; the only collective is one FP64 sum of the num and den tensors
when regions of one survey were spread over ranks.
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple


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
