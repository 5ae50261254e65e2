"""Factorised randoms (ck_set_randoms_factorised, Sec. 2.2, Eq. 7): the
randoms field computed from the angular and redshift selection instead of a
random catalog.  Against the oracle's FP64 evaluation (cells within float32
rounding, the zero pattern identical): a whole small box, and sampled cells
of the 512^3 survey grid; the field's total against N_tot (the densities are
normalised); the correlation sums against the oracle's with the same field;
determinism, independence of N_tot, an empty selection, and an argument
error that keeps the plan's previous randoms."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import Catalog, GridSpec, uniform_box, workload
from tests.gpu_util import cuda_torch, dev_cat, normwise, plan_for

pytestmark = pytest.mark.gpu

TOL = 1e-5
FIDUCIAL = dict(h0=100.0, omega_m=0.307, omega_k=0.0, omega_l=0.693, c=300000.0)  # Sec. 3


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _selection(seed, n_ra, n_dec, n_z, z_lo, z_hi, cut=True):
    """Random positive densities, a masked sky region, each normalised to
    integrate to 1 (per steradian over the sky, per unit z over [z_lo, z_hi))."""
    rng = np.random.default_rng(seed)
    pa = rng.uniform(0.3, 1.7, (n_dec, n_ra))
    if cut:
        pa[: n_dec // 3, :] = 0.0                 # the far south
        pa[:, 1: 1 + n_ra // 8] = 0.0             # a band in right ascension
    dec_e = np.radians(np.linspace(-90.0, 90.0, n_dec + 1))
    omega = (2.0 * np.pi / n_ra) * (np.sin(dec_e[1:]) - np.sin(dec_e[:-1]))
    pa /= float((pa * omega[:, None]).sum())
    pz = rng.uniform(0.5, 1.5, n_z)
    pz /= float(pz.sum() * (z_hi - z_lo) / n_z)
    return pa, pz


def _sel(pa, pz, z_lo, z_hi, z_max, n_tot=2.0e5):
    return dict(n_tot=n_tot, p_ang=pa, p_z=pz, z_lo=z_lo, z_hi=z_hi, z_max=z_max, **FIDUCIAL)


def _small():
    # a box beside the observer: x in [30, 270], |y| <= 100, |z| <= 90
    g = GridSpec((24, 20, 18), (30.0, -100.0, -90.0), 10.0, False)
    pa, pz = _selection(5, 36, 18, 4, 0.02, 0.11)
    return g, _sel(pa, pz, 0.02, 0.11, 0.13)


_SMALL_FIELD = {}


def _small_field():
    if "R" not in _SMALL_FIELD:
        g, sel = _small()
        _SMALL_FIELD["R"] = O.factorised_randoms(g, **sel)
    return _SMALL_FIELD["R"]


def _plan(g, shells, width, max_order, precision):
    from paper_2108_00015_gb300 import Plan
    return Plan(g.n, g.origin, g.cell, False, shells, width, max_order=max_order, precision=precision,
                padded=True)


def _set(plan, sel):
    kw = dict(sel)
    plan.set_randoms_factorised(kw.pop("n_tot"), kw.pop("p_ang"), kw.pop("p_z"), kw.pop("z_lo"), kw.pop("z_hi"),
                                **kw)


def _field(plan, g):
    R = plan.grids()[1].cpu().numpy().view(np.float32)
    return R[: g.n[2], : g.n[1], : g.n[0]].astype(np.float64)


def _close(got, want):
    """float32 cells: within 1e-6 relative of the oracle's FP64 values (the
    float32 evaluation's bound, 13 roundings of 2^-24 = 7.7e-7; cells near a
    bin edge are evaluated in FP64, within one rounding), and zeros exactly
    where the oracle has zeros (every bin decision is the FP64 one)."""
    assert np.array_equal(got == 0.0, want == 0.0), int(np.sum((got == 0.0) != (want == 0.0)))
    err = np.abs(got - want) / np.where(want != 0.0, np.abs(want), 1.0)
    assert float(err.max()) <= 1e-6, float(err.max())


def test_field_whole_box(torch):
    g, sel = _small()
    want = _small_field()
    assert (want > 0).sum() > 1000 and (want == 0).sum() > 500
    plan = _plan(g, (20.0, 30.0), 10.0, 2, "fp32")
    _set(plan, sel)
    _close(_field(plan, g), want)
    plan.close()



def test_field_on_bin_edges(torch):
    """Cell centres on the planes X = 0, Y = 0, Z = 0 (right ascension on
    its 0, 90, 180, 270 degree bin edges, declination 0 and the poles), the
    observer's own cell, and fine bins (0.5 degree, 50 redshift bins): many
    cells near an edge take the FP64 path; every decision must still be the
    oracle's.  (More near-edge cells than the FP64 queue holds for a box
    this size, so the FP64 kernel also takes its scan for marked cells.)"""
    g = GridSpec((25, 25, 25), (-150.0, -150.0, -150.0), 12.0, False)
    pa, pz = _selection(9, 720, 360, 50, 0.01, 0.08, cut=False)
    sel = _sel(pa, pz, 0.01, 0.08, 0.09)
    want = O.factorised_randoms(g, **sel)
    plan = _plan(g, (24.0, 36.0), 12.0, 2, "fp32")
    _set(plan, sel)
    got = _field(plan, g)
    assert got[12, 12, 12] == 0.0 and want[12, 12, 12] == 0.0     # r = 0
    _close(got, want)
    plan.close()


def test_survey_grid_sampled(torch):
    """The 512^3 survey grid (8 h^-1 Mpc cells around the observer), the
    plan bench.py times: sampled cells one by one against the oracle; the
    whole field's total against N_tot; two calls bit-identical."""
    w = workload("survey512", scale=0.01)
    g = w["grid"]
    pa, pz = _selection(7, 72, 36, 10, 0.2, 0.7)
    sel = _sel(pa, pz, 0.2, 0.7, 0.72, n_tot=8.0e5)
    plan = plan_for(w, max_order=3, precision="split_tf32")
    _set(plan, sel)
    R = plan.grids()[1].cpu().numpy().view(np.float32).astype(np.float64)
    # densities normalised: the field sums to N_tot (cells of 8 in a shell
    # 1100 thick; the sky cut's edges cost well under 1 %)
    assert abs(R.sum() / 8.0e5 - 1.0) < 0.01, R.sum()
    rng = np.random.default_rng(11)
    nz = np.argwhere(R > 0)
    pick = np.concatenate([nz[rng.integers(0, len(nz), 1200)],
                           np.stack([rng.integers(0, 512, 600) for _ in range(3)], axis=1)])
    cells = pick[:, ::-1]          # (iz, iy, ix) -> (ix, iy, iz)
    want = O.factorised_randoms_at(cells, g, **sel)
    got = R[pick[:, 0], pick[:, 1], pick[:, 2]]
    _close(got, want)
    # the same field again, bit for bit, and the same results
    res1 = plan.compute(*dev_cat(torch, w["data"]), orders=(2, 3), out="host")
    _set(plan, sel)
    R2 = plan.grids()[1].cpu().numpy().view(np.float32).astype(np.float64)
    assert np.array_equal(R, R2)
    res2 = plan.compute(*dev_cat(torch, w["data"]), orders=(2, 3), out="host")
    for n in (2, 3):
        assert np.array_equal(res1["xi"][n].numpy(), res2["xi"][n].numpy())
        assert np.all(np.isfinite(res1["xi"][n].numpy()))
    plan.close()


def _data(g, seed, n):
    L = np.array(g.n, np.float64) * g.cell
    c = uniform_box(seed, n, tuple(L))
    o = np.asarray(g.origin, np.float64)
    return Catalog((c.x + o[0]).astype(np.float32), (c.y + o[1]).astype(np.float32),
                   (c.z + o[2]).astype(np.float32))


@pytest.mark.parametrize("precision,orders", [("fp32", (2, 3)), ("split_tf32", (2, 3)), ("fp32", (2, 3, 4))])
def test_sums_vs_oracle(torch, precision, orders):
    g, sel = _small()
    R = _small_field()
    dat = _data(g, 13, 4000)
    shells, width = (20.0, 30.0, 40.0), 10.0
    ref = O.correlate(g, shells, width, dat, None, orders=orders, engine="direct", random_field=R)
    plan = _plan(g, shells, width, max(orders), precision)
    _set(plan, sel)
    res = plan.compute(*dev_cat(torch, dat), orders=orders, out="host")
    for n in orders:
        for key, akey in (("num", "abs_num"), ("den", "abs_den")):
            got = res[key][n].numpy()
            want = O.dense_tensor(ref[f"{key}{n}"], len(shells), n - 1)
            scale = O.dense_tensor(ref[f"{akey}{n}"], len(shells), n - 1)
            e = normwise(got, want, scale)
            assert e <= TOL, f"order {n} {key}: {e:.3e}"
    plan.close()


def test_n_tot_scale_free(torch):
    """alpha = data total / field total, so xi does not depend on N_tot
    (to float32 rounding of the cells)."""
    g, sel = _small()
    dat = _data(g, 17, 3000)
    plan = _plan(g, (20.0, 30.0), 10.0, 3, "fp32")
    out = []
    for n_tot in (2.0e5, 7.0e3):
        _set(plan, dict(sel, n_tot=n_tot))
        out.append(plan.compute(*dev_cat(torch, dat), orders=(2, 3), out="host"))
    for n in (2, 3):
        a, b = out[0]["xi"][n].numpy(), out[1]["xi"][n].numpy()
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5), (n, np.max(np.abs(a - b)))
    plan.close()


def test_empty_selection_and_bad_arguments(torch):
    from paper_2108_00015_gb300 import CkError
    g, sel = _small()
    dat = _data(g, 19, 2000)
    ran = _data(g, 20, 20000)
    plan = _plan(g, (20.0, 30.0), 10.0, 2, "fp32")
    # a selection that covers none of the box: no nonzero cell
    _set(plan, dict(sel, p_ang=np.zeros((18, 36))))
    with pytest.raises(CkError) as e:
        plan.compute(*dev_cat(torch, dat), orders=(2,), out="host")
    assert e.value.code == 12
    # an argument error leaves the previous randoms in place
    plan.set_randoms(*dev_cat(torch, ran))
    first = plan.compute(*dev_cat(torch, dat), orders=(2,), out="host")
    with pytest.raises(CkError) as e:
        _set(plan, dict(sel, z_lo=0.2, z_hi=0.1))
    assert e.value.code == 1
    again = plan.compute(*dev_cat(torch, dat), orders=(2,), out="host")
    assert np.array_equal(first["xi"][2].numpy(), again["xi"][2].numpy())
    plan.close()
