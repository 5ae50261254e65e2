"""The multi-rank host logic on CPU (gloo, world size 2): sharding of units
and the FP64 combination of per-region num / den (Eq. 19).  Each rank runs
the oracle on its own region; the combined result must equal the oracle on
the union of both regions."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle.conker_oracle as O
from paper_2108_00015_gb300.parallel import combine_regions, shard
from synth import GridSpec, lattice_catalog


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _regions():
    g = GridSpec((28, 12, 12), (0.0, 0.0, 0.0), 1.0, False)
    rng = np.random.default_rng(77)
    out = []
    for x0, nd, nr in ((1, 60, 400), (18, 50, 350)):
        cd = np.stack([rng.integers(x0, x0 + 8, nd), rng.integers(2, 10, nd), rng.integers(2, 10, nd)], 1)
        cr = np.stack([rng.integers(x0, x0 + 8, nr), rng.integers(2, 10, nr), rng.integers(2, 10, nr)], 1)
        out.append((lattice_catalog(g, cd), lattice_catalog(g, cr)))
    return g, out


SHELLS = ((1.5, 1.0), (2.5, 1.0), (3.2, 1.0))


def _sums(g, dat, ran):
    D, _ = O.grid_counts(dat.x, dat.y, dat.z, g)
    R, _ = O.grid_counts(ran.x, ran.y, ran.z, g)
    alpha, N, Rt = O.density_fields(D, R)
    offs = [O.shell_offsets(s, w, g.cell) for s, w in SHELLS]
    W = [O.convolve_direct(N, o, False) for o in offs]
    B = [O.convolve_direct(Rt, o, False) for o in offs]
    res = {}
    for n in (2, 3):
        res[n] = (O.product_sums(N, W, n)[0], O.product_sums(Rt, B, n)[0])
    return res


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, regions = _regions()
        mine = list(shard(len(regions), rank, world))
        num = {n: torch.zeros(len(O.multisets(3, n - 1)), dtype=torch.float64) for n in (2, 3)}
        den = {n: torch.zeros_like(num[n]) for n in (2, 3)}
        for i in mine:
            r = _sums(g, *regions[i])
            for n in (2, 3):
                num[n] += torch.from_numpy(r[n][0])
                den[n] += torch.from_numpy(r[n][1])
        cn, cd, cx = combine_regions(num, den)
        q.put((rank, {n: cn[n].numpy() for n in cn}, {n: cd[n].numpy() for n in cd}, {n: cx[n].numpy() for n in cx}))
    finally:
        dist.destroy_process_group()


def test_shard_covers_units():
    for n in (0, 1, 5, 16, 64):
        for w in (1, 2, 3, 8):
            got = [u for r in range(w) for u in shard(n, r, w)]
            assert got == list(range(n))


def test_two_rank_region_combination():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, regions = _regions()
    # the oracle on the union: both regions' separate fields summed (each with its own alpha)
    want = {}
    parts = [_sums(g, *reg) for reg in regions]
    for n in (2, 3):
        num = parts[0][n][0] + parts[1][n][0]
        den = parts[0][n][1] + parts[1][n][1]
        want[n] = (num, den, O.xi_from(num, den))
    for rank, num, den, xi in res:
        for n in (2, 3):
            assert np.allclose(num[n], want[n][0], rtol=1e-12, atol=0)
            assert np.allclose(den[n], want[n][1], rtol=1e-12, atol=0)
            assert np.allclose(xi[n], want[n][2], rtol=1e-12, atol=0)
