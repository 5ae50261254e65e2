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


SLAB_SHELLS = (1.5, 2.5)


def _slab_case():
    g = GridSpec((10, 9, 20), (0.0, 0.0, 0.0), 1.0, False)
    rng = np.random.default_rng(91)
    cd = np.stack([rng.integers(2, 8, 90), rng.integers(2, 7, 90), rng.integers(2, 18, 90)], 1)
    cr = np.stack([rng.integers(2, 8, 700), rng.integers(2, 7, 700), rng.integers(2, 18, 700)], 1)
    return g, lattice_catalog(g, cd), lattice_catalog(g, cr)


def _slab_worker(rank, world, port, q):
    """One slab per rank: select the slab's points on the host, agree on the
    whole catalog's alpha (all-reduce of the owned counts), sum the owned
    planes of the slab box (the oracle stands in for the library on a
    rank without a GPU) and combine through combine_regions."""
    from paper_2108_00015_gb300.parallel import global_alpha, in_planes, slab_box, slab_planes
    from synth import Catalog
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, data, rand = _slab_case()
        nz = g.n[2]
        halo = int(max(np.abs(O.shell_offsets(s, 1.0, g.cell))[:, 2].max() for s in SLAB_SHELLS))
        z0, z1 = slab_planes(nz, world, rank)
        lo, hi = slab_box(nz, z0, z1, halo)
        pick = lambda c, a, b: Catalog(*(v[in_planes(c.z, g.origin[2], g.cell, a, b)] for v in (c.x, c.y, c.z)))  # noqa: E731
        alpha = global_alpha(pick(data, z0, z1).n, pick(rand, z0, z1).n)
        gs = GridSpec((g.n[0], g.n[1], hi - lo), (g.origin[0], g.origin[1], g.origin[2] + lo * g.cell), g.cell, False)
        r = O.correlate(gs, SLAB_SHELLS, 1.0, pick(data, lo, hi), pick(rand, lo, hi), orders=(2, 3),
                        engine="direct", alpha=alpha, owned_z=(z0 - lo, z1 - lo))
        num = {n: torch.from_numpy(r[f"num{n}"]) for n in (2, 3)}
        den = {n: torch.from_numpy(r[f"den{n}"]) for n in (2, 3)}
        cn, cd, cx = combine_regions(num, den)
        q.put((rank, alpha, {n: cn[n].numpy() for n in cn}, {n: cd[n].numpy() for n in cd},
               {n: cx[n].numpy() for n in cx}))
    finally:
        dist.destroy_process_group()


def test_two_rank_slab_decomposition():
    """A catalog cut into two z slabs over two gloo ranks gives the undivided
    catalog's num, den and xi (Eq. 19 with the whole catalog's alpha)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, data, rand = _slab_case()
    whole = O.correlate(g, SLAB_SHELLS, 1.0, data, rand, orders=(2, 3), engine="direct")
    for rank, alpha, num, den, xi in res:
        assert alpha == pytest.approx(whole["alpha"], rel=1e-15)
        for n in (2, 3):
            assert np.allclose(num[n], whole[f"num{n}"], rtol=1e-12, atol=1e-9)
            assert np.allclose(den[n], whole[f"den{n}"], rtol=1e-12, atol=1e-9)
            assert np.allclose(xi[n], O.xi_from(whole[f"num{n}"], whole[f"den{n}"]), rtol=1e-11, atol=0)
