"""Seeded synthetic tracer catalogs shaped like a galaxy-survey workload.

The paper measures on SDSS DR12 CMASS galaxies, their randoms and
MultiDark-Patchy mocks (Sec. 3).  None of those are available here, so these
generators stand in for their shapes: clustered tracers (Neyman-Scott:
Poisson parents, Gaussian children), a lognormal-biased parent field, a
spherical-shell survey mask, and uniform randoms about 50 times denser.

Only positions are produced (float32, structure of arrays).  Every draw comes
from ``numpy.random.Generator(PCG64(seed))`` with the seed stated by the
caller; nothing here depends on the correlation method.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class GridSpec:
    """A cubic-cell grid: ``n`` cells per axis (x, y, z), lower corner
    ``origin``, cell side ``cell``; ``periodic`` selects a periodic box."""

    n: Tuple[int, int, int]
    origin: Tuple[float, float, float]
    cell: float
    periodic: bool

    @property
    def n_cells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    @property
    def length(self) -> Tuple[float, float, float]:
        return tuple(float(k) * self.cell for k in self.n)


@dataclasses.dataclass
class Catalog:
    """Point positions as float32 structure of arrays."""

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray

    def __post_init__(self):
        self.x = np.ascontiguousarray(self.x, dtype=np.float32)
        self.y = np.ascontiguousarray(self.y, dtype=np.float32)
        self.z = np.ascontiguousarray(self.z, dtype=np.float32)
        assert self.x.shape == self.y.shape == self.z.shape

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, idx) -> "Catalog":
        return Catalog(self.x[idx], self.y[idx], self.z[idx])

    @staticmethod
    def concat(cats: Sequence["Catalog"]) -> "Catalog":
        return Catalog(np.concatenate([c.x for c in cats]),
                       np.concatenate([c.y for c in cats]),
                       np.concatenate([c.z for c in cats]))


@dataclasses.dataclass(frozen=True)
class SurveyMask:
    """Observer at ``centre``; comoving distance in [r_min, r_max); a polar
    cap of half-angle ``cap_deg`` about +z (60 degrees = 25 % of the sky)."""

    centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    r_min: float = 1200.0
    r_max: float = 1800.0
    cap_deg: float = 60.0

    @property
    def cos_cap(self) -> float:
        return math.cos(math.radians(self.cap_deg))

    @property
    def volume(self) -> float:
        frac = (1.0 - self.cos_cap) / 2.0
        return frac * 4.0 / 3.0 * math.pi * (self.r_max ** 3 - self.r_min ** 3)

    def contains(self, x, y, z) -> np.ndarray:
        dx = np.asarray(x, np.float64) - self.centre[0]
        dy = np.asarray(y, np.float64) - self.centre[1]
        dz = np.asarray(z, np.float64) - self.centre[2]
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        with np.errstate(invalid="ignore", divide="ignore"):
            cz = np.where(r > 0, dz / np.where(r > 0, r, 1.0), 1.0)
        return (r >= self.r_min) & (r < self.r_max) & (cz >= self.cos_cap)

    def sample(self, rng: np.random.Generator, n: int):
        """Uniform points in the mask: r from the cube-root law, cos(theta)
        uniform in [cos_cap, 1], phi uniform in [0, 2 pi)."""
        u = rng.random(n)
        r = np.cbrt(u * (self.r_max ** 3 - self.r_min ** 3) + self.r_min ** 3)
        ct = self.cos_cap + (1.0 - self.cos_cap) * rng.random(n)
        phi = 2.0 * math.pi * rng.random(n)
        st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
        x = self.centre[0] + r * st * np.cos(phi)
        y = self.centre[1] + r * st * np.sin(phi)
        z = self.centre[2] + r * ct
        return x, y, z


def _to_periodic_f32(v: np.ndarray, length: float) -> np.ndarray:
    """Wrap float64 coordinates into [0, L) and round to float32; a value
    that rounds up to L is the same periodic point as 0."""
    v = np.mod(v, length)
    f = v.astype(np.float32)
    f[f >= np.float32(length)] = np.float32(0.0)
    return f


def _lengths(length) -> Tuple[float, float, float]:
    if np.ndim(length) == 0:
        return (float(length),) * 3
    return tuple(float(v) for v in length)


def uniform_box(seed: int, n: int, length) -> Catalog:
    """``n`` uniform points in the periodic box [0, L)^3 (or
    [0, Lx) x [0, Ly) x [0, Lz) for a triple of lengths)."""
    L = _lengths(length)
    rng = np.random.Generator(np.random.PCG64(seed))
    return Catalog(*(_to_periodic_f32(rng.random(n) * L[a], L[a]) for a in range(3)))


def neyman_scott_box(seed: int, n_parents: int, n_children: int, sigma: float,
                     length) -> Catalog:
    """Neyman-Scott process in a periodic box: Poisson (uniform) parents,
    each with exactly ``n_children`` children displaced by an isotropic
    Gaussian of ``sigma`` per axis, wrapped into the box.  Children of one
    parent are stored consecutively."""
    L = _lengths(length)
    rng = np.random.Generator(np.random.PCG64(seed))
    parents = rng.random((n_parents, 3)) * np.array(L)
    off = rng.normal(0.0, sigma, size=(n_parents, n_children, 3))
    pts = (parents[:, None, :] + off).reshape(-1, 3)
    return Catalog(*(_to_periodic_f32(pts[:, a], L[a]) for a in range(3)))


def uniform_survey(seed: int, n: int, mask: SurveyMask = SurveyMask(),
                   chunk: int = 1 << 24) -> Catalog:
    """``n`` uniform randoms inside the survey mask (direct sampling)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs, ys, zs = [], [], []
    left = n
    while left > 0:
        m = min(left, chunk)
        x, y, z = mask.sample(rng, m)
        xs.append(x.astype(np.float32))
        ys.append(y.astype(np.float32))
        zs.append(z.astype(np.float32))
        left -= m
    return Catalog(np.concatenate(xs), np.concatenate(ys), np.concatenate(zs))


def _gaussian_field(rng: np.random.Generator, m: int, box: float, k_cut: float) -> np.ndarray:
    """Unit-variance Gaussian random field on an m^3 grid over a periodic box
    of side ``box`` with power spectrum P(k) proportional to k^-2, cut to zero
    above ``k_cut``."""
    white = rng.normal(size=(m, m, m))
    k1 = 2.0 * math.pi * np.fft.fftfreq(m, d=box / m)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    sel = (k > 0) & (k <= k_cut)
    amp[sel] = 1.0 / k[sel]
    g = np.real(np.fft.ifftn(np.fft.fftn(white) * amp))
    g -= g.mean()
    s = g.std()
    return g / s if s > 0 else g


def continuous_maps(seed: int, shape, cell: float, sigma_g: float = 0.4, k_cut: float = 0.15,
                    footprint: float = 0.8):
    """A line-intensity-like pair of maps on a grid of ``shape`` (nz, ny, nx):
    a random-field map R, 1.0 to 2.0 inside an ellipsoidal footprint
    (semi-axes ``footprint`` times the half-box) and 0 outside, and a data map
    D = R exp(sigma_g G - sigma_g^2 / 2) with G a unit-variance Gaussian field
    (P(k) ~ k^-2 below ``k_cut`` h Mpc^-1).  Both float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = (int(v) for v in shape)
    white = rng.normal(size=(nz, ny, nx))
    kz, ky, kx = np.meshgrid(*[2.0 * math.pi * np.fft.fftfreq(m, d=cell) for m in (nz, ny, nx)], indexing="ij")
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    sel = (k > 0) & (k <= k_cut)
    amp[sel] = 1.0 / k[sel]
    g = np.real(np.fft.ifftn(np.fft.fftn(white) * amp))
    g = (g - g.mean()) / max(g.std(), 1e-300)
    zz, yy, xx = np.meshgrid(*[(np.arange(m) + 0.5) / m * 2.0 - 1.0 for m in (nz, ny, nx)], indexing="ij")
    rho2 = (xx * xx + yy * yy + zz * zz) / (footprint * footprint)
    R = np.where(rho2 < 1.0, 1.0 + rng.uniform(0.0, 1.0, (nz, ny, nx)), 0.0)
    D = R * np.exp(sigma_g * g - 0.5 * sigma_g * sigma_g)
    return D.astype(np.float32), R.astype(np.float32)


def neyman_scott_survey(seed: int, n_parents: int, n_children: int, sigma: float,
                        grid: GridSpec, mask: SurveyMask = SurveyMask(),
                        coarse: int = 64, sigma_g: float = 1.0) -> Catalog:
    """Neyman-Scott tracers in the survey mask with lognormal-biased parents.

    Parents are drawn uniformly in the mask and kept with probability
    proportional to exp(G - sigma_g^2 / 2), G a Gaussian field on a
    ``coarse``^3 grid over the box (P(k) ~ k^-2 below 2 pi / 64 h^-1 Mpc).
    Children are Gaussian about their parent; those that fall outside the
    mask are drawn again.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    box = grid.length[0]
    g = _gaussian_field(rng, coarse, box, 2.0 * math.pi / 64.0) * sigma_g
    dens = np.exp(g - 0.5 * sigma_g * sigma_g)
    dmax = float(dens.max())
    o = np.asarray(grid.origin, np.float64)
    cw = box / coarse
    px, py, pz = [], [], []
    have = 0
    while have < n_parents:
        m = max(4 * (n_parents - have), 1024)
        x, y, z = mask.sample(rng, m)
        ix = np.clip(((x - o[0]) // cw).astype(np.int64), 0, coarse - 1)
        iy = np.clip(((y - o[1]) // cw).astype(np.int64), 0, coarse - 1)
        iz = np.clip(((z - o[2]) // cw).astype(np.int64), 0, coarse - 1)
        keep = rng.random(m) * dmax < dens[iz, iy, ix]
        px.append(x[keep]); py.append(y[keep]); pz.append(z[keep])
        have += int(keep.sum())
    par = np.stack([np.concatenate(px)[:n_parents], np.concatenate(py)[:n_parents],
                    np.concatenate(pz)[:n_parents]], axis=1)
    pts = np.repeat(par, n_children, axis=0)
    out = pts + rng.normal(0.0, sigma, size=pts.shape)
    bad = ~mask.contains(out[:, 0], out[:, 1], out[:, 2])
    while bad.any():
        idx = np.nonzero(bad)[0]
        out[idx] = pts[idx] + rng.normal(0.0, sigma, size=(idx.size, 3))
        bad[idx] = ~mask.contains(out[idx, 0], out[idx, 1], out[idx, 2])
    return Catalog(out[:, 0], out[:, 1], out[:, 2])


def lattice_catalog(grid: GridSpec, cells: np.ndarray, mult: Optional[np.ndarray] = None,
                    where: str = "centre") -> Catalog:
    """Points placed exactly on chosen cells: ``cells`` is an int array
    [M, 3] of (ix, iy, iz); ``mult`` repeats each; ``where`` is "centre"
    (origin + (k + 1/2) g) or "edge" (origin + k g, the lower face)."""
    cells = np.asarray(cells, np.int64).reshape(-1, 3)
    if mult is not None:
        cells = np.repeat(cells, np.asarray(mult, np.int64), axis=0)
    f = 0.5 if where == "centre" else 0.0
    o = np.asarray(grid.origin, np.float64)
    pos = o[None, :] + (cells.astype(np.float64) + f) * grid.cell
    return Catalog(pos[:, 0], pos[:, 1], pos[:, 2])


# ---------------------------------------------------------------------------
# Named workloads (periodic 32^3 parity case, 512^3 survey, 256^3 stress).

def _shells(first: float, step: float, count: int):
    return tuple(float(first + step * i) for i in range(count))


SURVEY_GRID = GridSpec((512, 512, 512), (-2048.0, -2048.0, -2048.0), 8.0, False)

WORKLOADS: Dict[str, dict] = {
    # 320 h^-1 Mpc periodic box, 32^3 cells of 10; 5k clustered + 50k randoms.
    "periodic32": dict(
        grid=GridSpec((32, 32, 32), (0.0, 0.0, 0.0), 10.0, True),
        shells=(20.0, 40.0, 60.0, 80.0), width=10.0, orders=(2, 3),
        data=("ns_box", dict(seed=0, n_parents=250, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=1, n=50_000)),
    ),
    # 512^3 survey box of 8 h^-1 Mpc cells; 800k galaxies, 40M randoms;
    # 16 shells 30..150 in steps of 8, width 8.
    "survey512": dict(
        grid=SURVEY_GRID,
        shells=_shells(30.0, 8.0, 16), width=8.0, orders=(2, 3),
        data=("ns_survey", dict(seed=2, n_parents=40_000, n_children=20, sigma=8.0)),
        randoms=("uniform_survey", dict(seed=3, n=40_000_000)),
    ),
    # Same catalog, 32 shells 30..154 in steps of 4, width 4.
    "survey512_s32": dict(
        grid=SURVEY_GRID,
        shells=_shells(30.0, 4.0, 32), width=4.0, orders=(2, 3, 4),
        data=("ns_survey", dict(seed=2, n_parents=40_000, n_children=20, sigma=8.0)),
        randoms=("uniform_survey", dict(seed=3, n=40_000_000)),
    ),
    # Periodic 256^3 of 10 h^-1 Mpc; 20M clustered points, 40M randoms;
    # 16 shells 20..170 in steps of 10, width 10; orders up to 5.
    "stress256": dict(
        grid=GridSpec((256, 256, 256), (0.0, 0.0, 0.0), 10.0, True),
        shells=_shells(20.0, 10.0, 16), width=10.0, orders=(2, 3, 4, 5),
        data=("ns_box", dict(seed=4, n_parents=1_000_000, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=5, n=40_000_000)),
    ),
    # Small periodic case for profiler captures: 384^3 of 8 h^-1 Mpc (spectra
    # 228 MB, larger than L2), 4 shells, 50k clustered points, 2M randoms.
    "profile384": dict(
        grid=GridSpec((384, 384, 384), (0.0, 0.0, 0.0), 8.0, True),
        shells=(40.0, 60.0, 80.0, 100.0), width=8.0, orders=(2, 3),
        data=("ns_box", dict(seed=6, n_parents=2_500, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=7, n=2_000_000)),
    ),
    # Profiler case for the 16-shell contraction: periodic 256^3 of 10 h^-1
    # Mpc (W bank 1.07 GB per field), 50k clustered points, 2M randoms.
    "profile256s16": dict(
        grid=GridSpec((256, 256, 256), (0.0, 0.0, 0.0), 10.0, True),
        shells=_shells(20.0, 10.0, 16), width=10.0, orders=(2, 3),
        data=("ns_box", dict(seed=8, n_parents=2_500, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=9, n=2_000_000)),
    ),
    # Profiler case with the survey grid's transform lengths: periodic 512^3 of
    # 8 h^-1 Mpc, 2 shells (about 5 GB on the device), small catalogs.
    "profile512": dict(
        grid=GridSpec((512, 512, 512), (0.0, 0.0, 0.0), 8.0, True),
        shells=(40.0, 80.0), width=8.0, orders=(2, 3),
        data=("ns_box", dict(seed=10, n_parents=5_000, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=11, n=4_000_000)),
    ),
    # Profiler case for the fused last pass at the survey's x length and shell
    # count: periodic 512 x 128 x 128 of 8 h^-1 Mpc, the survey's 16 shells
    # (16 scratch spectra of 136 MB), small catalogs.
    "profile512x16": dict(
        grid=GridSpec((512, 128, 128), (0.0, 0.0, 0.0), 8.0, True),
        shells=_shells(30.0, 8.0, 16), width=8.0, orders=(2, 3),
        data=("ns_box", dict(seed=12, n_parents=2_500, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=13, n=2_000_000)),
    ),
    # Profiler case for the K^ z pass at the survey's z length and shell count:
    # periodic 128 x 256 x 512 of 8 h^-1 Mpc, the survey's 16 shells (16
    # scratch spectra of 71 MB, about 2 GB on the device), small catalogs.
    "profile_z512": dict(
        grid=GridSpec((128, 256, 512), (0.0, 0.0, 0.0), 8.0, True),
        shells=_shells(30.0, 8.0, 16), width=8.0, orders=(2, 3),
        data=("ns_box", dict(seed=14, n_parents=2_500, n_children=20, sigma=8.0)),
        randoms=("uniform_box", dict(seed=15, n=2_000_000)),
    ),
}


def _draw(kind: str, kw: dict, grid: GridSpec, scale: float) -> Catalog:
    kw = dict(kw)
    if kind == "ns_box":
        kw["n_parents"] = max(1, int(round(kw["n_parents"] * scale)))
        return neyman_scott_box(length=grid.length, **kw)
    if kind == "uniform_box":
        kw["n"] = max(1, int(round(kw["n"] * scale)))
        return uniform_box(length=grid.length, **kw)
    if kind == "ns_survey":
        kw["n_parents"] = max(1, int(round(kw["n_parents"] * scale)))
        return neyman_scott_survey(grid=grid, **kw)
    if kind == "uniform_survey":
        kw["n"] = max(1, int(round(kw["n"] * scale)))
        return uniform_survey(**kw)
    raise ValueError(kind)


def workload(name: str, scale: float = 1.0, with_points: bool = True) -> dict:
    """Return the named workload: grid, shells, width, orders and (unless
    ``with_points`` is False) the data and random catalogs.  ``scale``
    multiplies the number of parents / randoms (tests use small scales)."""
    w = dict(WORKLOADS[name])
    w["name"] = name
    if with_points:
        w["data"] = _draw(*w["data"], w["grid"], scale)
        w["randoms"] = _draw(*w["randoms"], w["grid"], scale)
    return w

# ---------------------------------------------------------------------------
# Batched workload: 64 mocks in 8 periodic grid classes (side, cell), 8 mocks
# per class, each with N_D log-uniform in [5e4, 2e6] points (20 children per
# Neyman-Scott parent, sigma uniform in [4, 12], seed 100 + i) and one
# uniform random catalog of 10M points per class (seed 200 + class); the
# survey's 16 shells; orders 2..4.

BATCH_CLASSES = ((128, 10.0), (160, 8.0), (192, 7.5), (240, 6.0), (256, 6.0), (288, 5.0), (320, 5.0), (384, 5.0))


def batch_workload(scale: float = 1.0, mocks_per_class: int = 8, n_randoms: int = 10_000_000) -> dict:
    """Grid classes with their randoms and the mocks as (class index, Catalog);
    ``scale`` multiplies the point counts."""
    classes = []
    for c, (n, cell) in enumerate(BATCH_CLASSES):
        g = GridSpec((n, n, n), (0.0, 0.0, 0.0), cell, True)
        classes.append(dict(grid=g, randoms=uniform_box(200 + c, max(1, int(round(n_randoms * scale))), g.length)))
    mocks = []
    for i in range(len(BATCH_CLASSES) * mocks_per_class):
        c = i // mocks_per_class
        rng = np.random.Generator(np.random.PCG64(100 + i))
        n_d = math.exp(rng.uniform(math.log(5e4), math.log(2e6))) * scale
        sigma = rng.uniform(4.0, 12.0)
        g = classes[c]["grid"]
        mocks.append((c, neyman_scott_box(100 + i, max(1, int(round(n_d / 20))), 20, sigma, g.length)))
    return dict(name="batch64", classes=classes, mocks=mocks, shells=_shells(30.0, 8.0, 16), width=8.0,
                orders=(2, 3, 4))
