"""The seeded generators: determinism and the shape of the workloads."""
import numpy as np

from synth import SurveyMask, neyman_scott_box, neyman_scott_survey, uniform_box, uniform_survey, workload
from synth.catalogs import SURVEY_GRID


def test_deterministic():
    a = neyman_scott_box(0, 50, 20, 8.0, 320.0)
    b = neyman_scott_box(0, 50, 20, 8.0, 320.0)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.z, b.z)
    assert a.n == 1000 and a.x.dtype == np.float32


def test_periodic_range():
    c = uniform_box(1, 20000, 320.0)
    for v in (c.x, c.y, c.z):
        assert v.min() >= 0 and v.max() < np.float32(320.0)


def test_survey_in_mask():
    m = SurveyMask()
    r = uniform_survey(3, 20000)
    assert m.contains(r.x, r.y, r.z).mean() > 0.999  # float32 rounding at the edges
    d = neyman_scott_survey(2, 200, 20, 8.0, SURVEY_GRID)
    assert d.n == 4000 and m.contains(d.x, d.y, d.z).mean() > 0.999
    assert abs(m.volume - 4.298e9) / 4.298e9 < 1e-3


def test_workload_scaled():
    w = workload("periodic32")
    assert w["data"].n == 5000 and w["randoms"].n == 50000
    assert w["grid"].n == (32, 32, 32)


def test_continuous_maps():
    """Seeded maps: the same arrays for the same seed; R is 1..2 inside the
    footprint and 0 outside; D is non-negative and 0 where R is 0."""
    from synth import continuous_maps
    a = continuous_maps(4, (12, 10, 8), 10.0)
    b = continuous_maps(4, (12, 10, 8), 10.0)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    D, R = a
    assert D.shape == R.shape == (12, 10, 8) and D.dtype == R.dtype == np.float32
    inside = R > 0
    assert 0.1 < inside.mean() < 0.9
    assert float(R[inside].min()) >= 1.0 and float(R[inside].max()) <= 2.0
    assert float(D.min()) >= 0.0 and float(np.abs(D[~inside]).max()) == 0.0
