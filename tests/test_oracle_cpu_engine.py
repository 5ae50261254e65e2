"""The FP64 C++/OpenMP engine (oracle/conker_cpu.cpp) against the pinned
numpy oracle on small grids: the same mapping, convolution (direct and FFT)
and product sums, to 1e-12 of the sums of |terms|, for periodic and survey
boxes, both shell rules, every order, and a region of a decomposed catalog
(the whole catalog's alpha, owned planes).  CPU only."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from oracle import cpu_engine as C
from synth import GridSpec, lattice_catalog, neyman_scott_box, uniform_box


def _close(a, b, scale, tol=1e-12):
    return np.all(np.abs(a - b) <= tol * np.maximum(scale, 1e-300))


def _compare(g, shells, width, data, rand, orders, engine, rule="center_bin", **kw):
    want = O.correlate(g, shells, width, data, rand, orders=orders, engine=engine, rule=rule, **kw)
    got = C.correlate(g, shells, width, data, rand, orders=orders, engine=engine, rule=rule, **kw)
    assert got["alpha"] == pytest.approx(want["alpha"], rel=1e-15)
    assert (got["dropped_d"], got["dropped_r"]) == (want["dropped_d"], want["dropped_r"])
    for n in orders:
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            assert _close(got[f"{key}{n}"], want[f"{key}{n}"], want[f"{akey}{n}"]), f"{engine} order {n} {key}"
            assert _close(got[f"{akey}{n}"], want[f"{akey}{n}"], want[f"{akey}{n}"]), f"{engine} order {n} {akey}"


@pytest.mark.parametrize("engine", ["direct", "fft"])
def test_periodic_all_orders(engine):
    g = GridSpec((16, 12, 10), (0.0, 0.0, 0.0), 1.0, True)
    L = (16.0, 12.0, 10.0)
    data = neyman_scott_box(3, 40, 8, 1.0, L)
    rand = uniform_box(4, 4000, L)
    _compare(g, (1.5, 2.5, 3.0), 1.0, data, rand, (2, 3, 4, 5), engine)


def test_intersect_rule_and_lengths_3_5():
    g = GridSpec((15, 18, 20), (0.0, 0.0, 0.0), 2.0, True)
    L = (30.0, 36.0, 40.0)
    data = neyman_scott_box(5, 30, 6, 2.0, L)
    rand = uniform_box(6, 3000, L)
    for engine in ("direct", "fft"):
        _compare(g, (3.0, 5.0), 0.0, data, rand, (2, 3), engine, rule="intersect")


def test_survey_box_and_region():
    g = GridSpec((16, 12, 20), (-7.0, 3.0, 0.0), 1.0, False)
    rng = np.random.default_rng(8)
    cd = np.stack([rng.integers(3, 11, 80), rng.integers(3, 9, 80), rng.integers(3, 17, 80)], 1)
    cr = np.stack([rng.integers(3, 11, 600), rng.integers(3, 9, 600), rng.integers(3, 17, 600)], 1)
    data, rand = lattice_catalog(g, cd), lattice_catalog(g, cr)
    for engine in ("direct", "fft"):
        _compare(g, (1.5, 2.5), 1.0, data, rand, (2, 3, 4), engine)
    _compare(g, (1.5, 2.5), 1.0, data, rand, (2, 3), "direct", alpha=0.1, owned_z=(5, 12))
