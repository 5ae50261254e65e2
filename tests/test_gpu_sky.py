"""Survey input (ck_sky_to_cartesian, Sec. 2.2, Eqs. 3-6): the device's
distance table and coordinates against the oracle's FP64 quadrature and
Eqs. 4-6 (float32 outputs within two units in the last place of r), in the
paper's fiducial cosmology (Sec. 3) and an open one; the Einstein-de Sitter
closed form; out-of-range redshifts and non-finite angles give NaN, which
the gridding drops and counts."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from synth import GridSpec
from tests.gpu_util import cuda_torch, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_torch()


def _sky(seed, n, zlo=0.43, zhi=0.7):
    rng = np.random.default_rng(seed)
    ra = rng.uniform(0.0, 360.0, n).astype(np.float32)
    dec = np.degrees(np.arcsin(rng.uniform(-0.5, 0.95, n))).astype(np.float32)
    z = rng.uniform(zlo, zhi, n).astype(np.float32)
    return ra, dec, z


@pytest.mark.parametrize("cosmo", [
    dict(h0=100.0, omega_m=0.307, omega_k=0.0, omega_l=0.693, c=300000.0),     # Sec. 3
    dict(h0=67.7, omega_m=0.31, omega_k=0.05, omega_l=0.64, c=299792.458),
])
def test_sky_vs_oracle(torch, cosmo):
    from paper_2108_00015_gb300 import sky_to_cartesian
    ra, dec, z = _sky(1, 3000)
    X, Y, Z = sky_to_cartesian(dev(torch, ra), dev(torch, dec), dev(torch, z), z_max=0.75, **cosmo)
    wx, wy, wz = O.sky_to_cartesian(ra, dec, z, cosmo["h0"], cosmo["omega_m"], cosmo["omega_k"],
                                    cosmo["omega_l"], cosmo["c"])
    r = np.sqrt(wx ** 2 + wy ** 2 + wz ** 2)
    ulp = np.spacing(r.astype(np.float32)).astype(np.float64)
    for got, want in ((X, wx), (Y, wy), (Z, wz)):
        err = np.abs(got.cpu().numpy().astype(np.float64) - want)
        assert np.all(err <= 2 * ulp), float(np.max(err / ulp))


def test_sky_closed_form(torch):
    """Einstein-de Sitter (O_M = 1): r = 2 (c/H0) (1 - 1/sqrt(1+z)), over 0 <= z <= 3."""
    from paper_2108_00015_gb300 import sky_to_cartesian
    z = np.linspace(0.0, 3.0, 2001).astype(np.float32)
    ra = np.zeros_like(z)
    dec = np.zeros_like(z)
    X, Y, Z = sky_to_cartesian(dev(torch, ra), dev(torch, dec), dev(torch, z), h0=70.0, omega_m=1.0,
                               omega_k=0.0, omega_l=0.0, c=299792.458, z_max=3.0)
    want = 2.0 * 299792.458 / 70.0 * (1.0 - 1.0 / np.sqrt(1.0 + z.astype(np.float64)))
    got = X.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - want) <= np.spacing(want.astype(np.float32)) + 1e-30)
    assert float(np.abs(Y.cpu().numpy()).max()) == 0.0 and float(np.abs(Z.cpu().numpy()).max()) == 0.0


def test_sky_out_of_range_dropped(torch):
    """Redshifts outside [0, z_max] and non-finite angles give NaN
    coordinates; a plan drops and counts those points."""
    from paper_2108_00015_gb300 import Plan, sky_to_cartesian
    ra, dec, z = _sky(2, 4000, 0.45, 0.6)
    z[:10] = -0.1
    z[10:20] = 0.9
    ra[20] = np.nan
    dec[21] = np.inf
    X, Y, Z = sky_to_cartesian(dev(torch, ra), dev(torch, dec), dev(torch, z), z_max=0.8)
    bad = np.isnan(X.cpu().numpy())
    assert bad.sum() == 22 and bad[:22].all()
    # a grid around the survey (padded: the points reach its faces)
    g = GridSpec((128, 128, 128), (-1700.0, -1700.0, -1700.0), 27.0, False)
    plan = Plan(g.n, g.origin, g.cell, False, (60.0, 90.0), 27.0, max_order=2, padded=True)
    plan.set_randoms(X, Y, Z)
    res = plan.compute(X, Y, Z, orders=(2,), out="host")
    assert res["dropped"].numpy().tolist() == [22, 22]
    D, R = plan.grids()
    assert int(D.sum()) == 4000 - 22 and int(R.sum()) == 4000 - 22
    plan.close()
