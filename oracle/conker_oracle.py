"""Plain FP64 CPU oracle for ConKer's hot path (arXiv 2108.00015).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The library
(C-ABI + CUDA kernels) never imports, links or calls it, and it shares no code,
table or constant with that library.

What it computes, in the paper's order and notation (Sec. 2):

* mapping (Sec. 2.2): histograms D, R of tracer counts per cubic cell of side
  g_s; R normalised to the data total, alpha = sum D / sum R; the density
  variation N = D - alpha R (Eq. 8) and the normalised random field
  Rt = alpha R;
* kernels (Sec. 2.3): the spherical-shell kernel K_s as a list of integer cell
  offsets m (K_s(m) = 1 on the list, 0 elsewhere);
* convolution (Sec. 2.4): W_s(r) = sum_m K_s(m) N(r + m) (Eq. 9, the inner
  product of the kernel centred on cell r with N), B_s the same for Rt
  (Eq. 10), and W_0 = N, B_0 = Rt;
* summation (Sec. 2.5): for every multiset s_1 <= ... <= s_{n-1}
  num = sum_r W_0 prod_i W_{s_i}, den = sum_r B_0 prod_i B_{s_i},
  xi_n = num / den (Eqs. 11-13); the equidistant diagonal (Eq. 14).

Equation numbers count the paper's numbered displays in order:
(1) Delta, (2) the xi_n integral, (3) r(z), (4)-(6) X, Y, Z, (7) factorised
randoms, (8) N = D - R, (9) W_i = N***K_i, (10) B_i = R***K_i, (11) xi_n,
(12) xi_2, (13) xi_3, (14) xi_n diagonal, (15)-(17) continuous field,
(18) Landy-Szalay, (19) combined regions.

Readings where the paper is silent or ambiguous (each is a choice):

1. Cell assignment (Sec. 2.2 says "histogram"): nearest-grid-point; a point x
   is in cell k of an axis iff e_k <= x < e_{k+1} with the edge
   e_k = fl64(origin + fl64(k * g)) compared exactly against the float32
   coordinate.  Periodic grids take k mod n; otherwise points with k outside
   [0, n) are dropped and counted.
2. Shell membership (Sec. 2.3, "cells intersected by a sphere of radius s_i",
   and the bins of width w of Sec. 3): rule "center_bin" (default) keeps the
   offset m iff (s - w/2) <= |m| g < (s + w/2), distances between cell
   centres, compared as squares in FP64; rule "intersect" keeps m iff the
   sphere of radius s meets the closed cell cube: dmin^2 <= s^2 < dmax^2.
3. The kernel cube is centred on a cell (Fig. 3 puts the result in the
   centre cell), so offsets run over all integer m, not a cube of even side.
4. Boundaries: a periodic grid uses circular index arithmetic (valid while
   2 max|m_i| < n_i); a non-periodic grid treats cells outside the box as 0.
5. alpha = sum D / sum R over the histograms (the data total N_tot of
   Sec. 2.2 counts the gridded points).
6. Multisets with repetition (the diagonal of Eq. 14 is part of the tensor).
7. A non-positive denominator gives xi = NaN for that entry.
8. Weighted histograms (Sec. 2.2 allows "weighted counts"; Sec. 3 uses the
   survey's systematic and FKP weights): a cell holds the sum of its points'
   weights, each weight rounded to the nearest multiple of 2^-32 (ties to
   even), summed exactly; a point with a non-finite weight is dropped.  The
   rounding makes the sums independent of the order of addition; it moves a
   weight by at most 2^-33.
9. Sky coordinates (Sec. 2.2): right ascension and declination in degrees;
   r(z) is Eq. 3's line-of-sight integral exactly as printed (no curvature
   transform), and X, Y, Z follow Eqs. 4-6.
10. Factorised randoms (Eq. 7): P_ang is a probability per steradian on an
   equiangular grid of right ascension [0, 360) x declination [-90, 90]
   (nearest cell), P_z a probability per unit redshift in uniform bins of
   [z_lo, z_hi) (0 outside); the expected count of a grid cell is the
   density at its centre times its volume,
   R = N_tot P_ang(ra, dec) P_z(z(r)) (dz/dr) g^3 / r^2, dz/dr = H0 E(z) / c,
   and 0 where r exceeds r(z_max) or r = 0.
11. Continuous fields (Sec. 2.7, Eqs. 15-17): delta = (D - R) / R per cell
   where R > 0 and 0 where R <= 0 (no survey there); W_0 = delta,
   W_s = delta *** K_s and xi_n = sum_r W_0 prod W_{s_i}, no denominator.
12. Cross-correlation (Sec. 2.8): W_0 = Delta_0, W_s = Delta_1 *** K_s, the
   sums of Eq. 16 (xi_2 of Eq. 17 and, by the same product, higher orders).
13. Per-cell maps (Sec. 4.2, the wishbone and sky-slice figures):
   W_0 W_s / <B_0 B_s> per cell, the average over the box's cells,
   <B_0 B_s> = den_2(s) / N_box.
14. Regions of one catalog (Sec. 4's combination of the two galactic caps,
   Eq. 19, adds numerators and denominators before dividing): a catalog cut
   into slabs along z sums each slab's owned planes with every field of the
   slab box, halo planes included, in the convolution, and with the whole
   catalog's alpha, so that the slabs' num and den add to the whole's.

Pins: see tests/test_oracle_pins.py (brute-force pair and triplet counts on
cell-centred points, three-square lattice counts, closed forms, symmetry,
translation invariance, linearity, region additivity, direct vs FFT engine).
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, Iterable, List, Sequence, Tuple

import numpy as np

__all__ = [
    "cell_edge", "cell_index", "grid_counts", "grid_weights", "quantize_weights", "density_fields", "shell_offsets",
    "check_periodic_support", "kernel_grid", "convolve_direct", "convolve_fft",
    "w_at_cells", "multisets", "product_sums", "dense_tensor", "xi_from",
    "xi_diagonal", "correlate", "kernel_spectrum_octant", "guard_band_ok", "pair_sums_fft",
    "comoving_distance", "sky_to_cartesian", "factorised_randoms_at", "factorised_randoms",
    "delta_field", "field_sums", "product_map",
]


# ---------------------------------------------------------------------------
# Mapping (Sec. 2.2, Eq. 8)

def cell_edge(origin: float, cell: float, k) -> np.ndarray:
    """Lower edge of cell k on one axis: fl64(origin + fl64(k * cell))."""
    k = np.asarray(k, dtype=np.float64)
    return np.float64(origin) + k * np.float64(cell)


def cell_index(x: np.ndarray, origin: float, cell: float) -> np.ndarray:
    """The unique integer k with cell_edge(k) <= x < cell_edge(k + 1)
    (reading 1), for float32 coordinates ``x``; returns int64."""
    xd = np.asarray(x, dtype=np.float32).astype(np.float64)
    k = np.floor((xd - origin) / cell).astype(np.int64)
    for _ in range(8):
        lo = xd < cell_edge(origin, cell, k)
        hi = xd >= cell_edge(origin, cell, k + 1)
        if not (lo.any() or hi.any()):
            return k
        k = k - lo.astype(np.int64) + hi.astype(np.int64)
    raise AssertionError("cell_index did not settle")


def grid_counts(x, y, z, grid) -> Tuple[np.ndarray, int]:
    """Histogram of points per cell, shape (nz, ny, nx) uint32, and the number
    of points dropped outside a non-periodic grid (Sec. 2.2, reading 1)."""
    nx, ny, nz = (int(v) for v in grid.n)
    ks = []
    for coord, o, n in ((x, grid.origin[0], nx), (y, grid.origin[1], ny), (z, grid.origin[2], nz)):
        k = cell_index(coord, o, grid.cell)
        ks.append(np.mod(k, n) if grid.periodic else k)
    kx, ky, kz = ks
    if grid.periodic:
        keep = np.ones(kx.shape, dtype=bool)
    else:
        keep = (kx >= 0) & (kx < nx) & (ky >= 0) & (ky < ny) & (kz >= 0) & (kz < nz)
    dropped = int(kx.size - int(keep.sum()))
    flat = (kz[keep] * ny + ky[keep]) * nx + kx[keep]
    counts = np.bincount(flat, minlength=nx * ny * nz)
    assert counts.max(initial=0) < 2 ** 32
    return counts.astype(np.uint32).reshape(nz, ny, nx), dropped


WEIGHT_FRAC_BITS = 32


def quantize_weights(w) -> np.ndarray:
    """Reading 8: each weight as an integer count of 2^-32 (nearest, ties to
    even).  The product of a float32 weight and 2^32 is exact in FP64."""
    return np.rint(np.asarray(w, np.float32).astype(np.float64) * 2.0 ** WEIGHT_FRAC_BITS).astype(np.int64)


def grid_weights(x, y, z, w, grid) -> Tuple[np.ndarray, float, int]:
    """Weighted histogram (Sec. 2.2, reading 8): per cell the exact sum of the
    kept points' rounded weights, as FP64 of shape (nz, ny, nx); the total of
    those weights; and the number of dropped points (outside a non-periodic
    grid, or with a non-finite weight)."""
    nx, ny, nz = (int(v) for v in grid.n)
    w = np.asarray(w, np.float32)
    ks = []
    for coord, o, n in ((x, grid.origin[0], nx), (y, grid.origin[1], ny), (z, grid.origin[2], nz)):
        k = cell_index(coord, o, grid.cell)
        ks.append(np.mod(k, n) if grid.periodic else k)
    kx, ky, kz = ks
    keep = np.isfinite(w)
    if not grid.periodic:
        keep &= (kx >= 0) & (kx < nx) & (ky >= 0) & (ky < ny) & (kz >= 0) & (kz < nz)
    dropped = int(w.size - int(keep.sum()))
    flat = (kz[keep] * ny + ky[keep]) * nx + kx[keep]
    q = quantize_weights(w[keep])
    sums = np.zeros(nx * ny * nz, np.int64)
    np.add.at(sums, flat, q)
    assert np.abs(sums).max(initial=0) < 2 ** 53
    scale = 2.0 ** -WEIGHT_FRAC_BITS
    return (sums.astype(np.float64) * scale).reshape(nz, ny, nx), float(int(q.sum())) * scale, dropped


def density_fields(D: np.ndarray, R: np.ndarray, alpha: float = None):
    """alpha = sum D / sum R, N = D - alpha R (Eq. 8 with R normalised to the
    data total, Sec. 2.2) and Rt = alpha R, all FP64.  A given alpha (the
    whole catalog's, for one region of it: reading 14) replaces the ratio."""
    sd = float(np.sum(D, dtype=np.float64))
    sr = float(np.sum(R, dtype=np.float64))
    if alpha is None:
        if sr <= 0.0:
            raise ValueError("random histogram is empty")
        alpha = sd / sr
    alpha = float(alpha)
    Dd = D.astype(np.float64)
    Rd = R.astype(np.float64)
    return alpha, Dd - alpha * Rd, alpha * Rd


# ---------------------------------------------------------------------------
# Input coordinates (Sec. 2.2, Eqs. 3-6)

def comoving_distance(z, h0: float, omega_m: float, omega_k: float, omega_l: float, c: float) -> np.ndarray:
    """Eq. 3: r(z) = (c / H0) int_0^z dz' / sqrt(O_M (1+z')^3 + O_k (1+z')^2 + O_L),
    by adaptive quadrature (a library primitive) for every redshift, FP64."""
    from scipy.integrate import quad
    z = np.asarray(z, np.float64)
    f = lambda t: 1.0 / math.sqrt(omega_m * (1 + t) ** 3 + omega_k * (1 + t) ** 2 + omega_l)  # noqa: E731
    out = np.empty(z.shape, np.float64)
    for i, zi in np.ndenumerate(z):
        out[i] = (c / h0) * quad(f, 0.0, float(zi), epsabs=0.0, epsrel=1e-13, limit=200)[0]
    return out


def sky_to_cartesian(ra_deg, dec_deg, z, h0: float, omega_m: float, omega_k: float, omega_l: float,
                     c: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Eqs. 4-6: X = r cos(dec) cos(ra), Y = r cos(dec) sin(ra), Z = r sin(dec),
    r = r(z) of Eq. 3, angles in degrees (reading 9), FP64."""
    r = comoving_distance(z, h0, omega_m, omega_k, omega_l, c)
    a = np.radians(np.asarray(ra_deg, np.float64))
    d = np.radians(np.asarray(dec_deg, np.float64))
    return r * np.cos(d) * np.cos(a), r * np.cos(d) * np.sin(a), r * np.sin(d)


def factorised_randoms_at(cells, grid, n_tot: float, p_ang: np.ndarray, p_z: np.ndarray, z_lo: float, z_hi: float,
                          z_max: float, h0: float, omega_m: float, omega_k: float, omega_l: float,
                          c: float) -> np.ndarray:
    """Eq. 7 (reading 10) at chosen cells (ix, iy, iz) of the grid, FP64:
    p_ang has shape (n_dec, n_ra), p_z shape (n_z,).  z(r) inverts Eq. 3 by
    root finding (a library primitive)."""
    from scipy.optimize import brentq
    cells = np.asarray(cells, np.int64).reshape(-1, 3)
    ctr = np.asarray(grid.origin, np.float64) + (cells + 0.5) * grid.cell
    X, Y, Z = ctr[:, 0], ctr[:, 1], ctr[:, 2]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rmax = float(comoving_distance(z_max, h0, omega_m, omega_k, omega_l, c))
    n_dec, n_ra = p_ang.shape
    out = np.zeros(len(cells), np.float64)
    for i in range(len(cells)):
        if not (0.0 < r[i] <= rmax):
            continue
        zi = brentq(lambda t: float(comoving_distance(t, h0, omega_m, omega_k, omega_l, c)) - r[i], 0.0, z_max,
                    xtol=1e-14, rtol=1e-14)
        if not (z_lo <= zi < z_hi):
            continue
        ra = math.degrees(math.atan2(Y[i], X[i])) % 360.0
        dec = math.degrees(math.asin(Z[i] / r[i]))
        ia = min(int(ra / 360.0 * n_ra), n_ra - 1)
        idd = min(int((dec + 90.0) / 180.0 * n_dec), n_dec - 1)
        iz = min(int((zi - z_lo) / (z_hi - z_lo) * len(p_z)), len(p_z) - 1)
        a = 1.0 + zi
        dzdr = h0 * math.sqrt(omega_m * a ** 3 + omega_k * a ** 2 + omega_l) / c
        out[i] = n_tot * float(p_ang[idd, ia]) * float(p_z[iz]) * dzdr * grid.cell ** 3 / (r[i] * r[i])
    return out


def factorised_randoms(grid, **sel) -> np.ndarray:
    """The whole randoms field of Eq. 7, shape (nz, ny, nx), FP64."""
    nx, ny, nz = grid.n
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
    return factorised_randoms_at(cells, grid, **sel).reshape(nz, ny, nx)


# ---------------------------------------------------------------------------
# Kernels (Sec. 2.3)

def shell_offsets(radius: float, width: float, cell: float, rule: str = "center_bin") -> np.ndarray:
    """Integer offsets m = (mx, my, mz) with K_s(m) = 1 (readings 2 and 3),
    int64 array [M, 3] in lexicographic (mx, my, mz) order."""
    g2 = np.float64(cell) * np.float64(cell)
    if rule == "center_bin":
        outer = radius + 0.5 * width
    elif rule == "intersect":
        outer = radius + cell
    else:
        raise ValueError(rule)
    h = int(math.ceil(outer / cell)) + 1
    r = np.arange(-h, h + 1, dtype=np.int64)
    mx, my, mz = np.meshgrid(r, r, r, indexing="ij")
    mx, my, mz = mx.ravel(), my.ravel(), mz.ravel()
    if rule == "center_bin":
        lo = max(radius - 0.5 * width, 0.0)
        hi = radius + 0.5 * width
        d2 = (mx * mx + my * my + mz * mz).astype(np.float64) * g2
        sel = (d2 >= np.float64(lo) * np.float64(lo)) & (d2 < np.float64(hi) * np.float64(hi))
    else:
        def near(a):
            t = np.maximum(np.abs(a).astype(np.float64) - 0.5, 0.0)
            return t * t
        def far(a):
            t = np.abs(a).astype(np.float64) + 0.5
            return t * t
        dmin2 = (near(mx) + near(my) + near(mz)) * g2
        dmax2 = (far(mx) + far(my) + far(mz)) * g2
        s2 = np.float64(radius) * np.float64(radius)
        sel = (dmin2 <= s2) & (s2 < dmax2)
    return np.stack([mx[sel], my[sel], mz[sel]], axis=1)


def check_periodic_support(offsets: np.ndarray, n: Sequence[int]) -> bool:
    """Reading 4: on a periodic axis of n cells, distinct offsets stay
    distinct after wrapping iff 2 max|m| < n."""
    if offsets.size == 0:
        return True
    m = np.abs(offsets).max(axis=0)
    return bool(all(2 * int(m[a]) < int(n[a]) for a in range(3)))


def kernel_grid(offsets: np.ndarray, n: Sequence[int]) -> np.ndarray:
    """K_s on the full (nz, ny, nx) grid with offsets wrapped periodically."""
    nx, ny, nz = (int(v) for v in n)
    K = np.zeros((nz, ny, nx), dtype=np.float64)
    np.add.at(K, (np.mod(offsets[:, 2], nz), np.mod(offsets[:, 1], ny),
                  np.mod(offsets[:, 0], nx)), 1.0)
    return K


def kernel_spectrum_octant(offsets: np.ndarray, n: Sequence[int]) -> np.ndarray:
    """The discrete Fourier transform of K_s on the grid, divided by N_c,
    on the octant 0 <= k_a <= n_a/2 (shape (nz/2+1, ny/2+1, nx/2+1)).  K_s is
    even in every axis, so its transform is real and even in every axis."""
    nx, ny, nz = (int(v) for v in n)
    K = kernel_grid(offsets, n)
    Kh = np.fft.rfftn(K).real / float(nx * ny * nz)
    return Kh[: nz // 2 + 1, : ny // 2 + 1, : nx // 2 + 1]


# ---------------------------------------------------------------------------
# Convolution (Sec. 2.4, Eqs. 9-10)

def _shift_zero(F: np.ndarray, m: Tuple[int, int, int]) -> np.ndarray:
    """G(r) = F(r + m) with zeros outside the box (non-periodic grid)."""
    out = np.zeros_like(F)
    src = []
    dst = []
    for axis, mm in ((0, m[2]), (1, m[1]), (2, m[0])):
        n = F.shape[axis]
        if abs(mm) >= n:
            return out
        if mm >= 0:
            src.append(slice(mm, n)); dst.append(slice(0, n - mm))
        else:
            src.append(slice(0, n + mm)); dst.append(slice(-mm, n))
    out[tuple(dst)] = F[tuple(src)]
    return out


def convolve_direct(F: np.ndarray, offsets: np.ndarray, periodic: bool) -> np.ndarray:
    """W(r) = sum over the kernel's offsets m of F(r + m): the inner product of
    the kernel centred on cell r with the field (Eq. 9 / Eq. 10), evaluated
    directly in real space.  F has shape (nz, ny, nx)."""
    W = np.zeros(F.shape, dtype=np.float64)
    for mx, my, mz in offsets:
        if periodic:
            W += np.roll(F, shift=(-int(mz), -int(my), -int(mx)), axis=(0, 1, 2))
        else:
            W += _shift_zero(F, (int(mx), int(my), int(mz)))
    return W


def convolve_fft(F: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """The same inner product by FFT (periodic grid): the correlation
    theorem, W = IFFT( FFT(F) * conj(FFT(K)) ), with a library FFT in FP64."""
    n = (F.shape[2], F.shape[1], F.shape[0])
    K = kernel_grid(offsets, n)
    return np.fft.irfftn(np.fft.rfftn(F) * np.conj(np.fft.rfftn(K)), s=F.shape, axes=(0, 1, 2))


def w_at_cells(F: np.ndarray, offsets: np.ndarray, cells: np.ndarray, periodic: bool) -> np.ndarray:
    """W(r) at chosen cells r = (ix, iy, iz), one by one (direct sum)."""
    nz, ny, nx = F.shape
    cells = np.asarray(cells, np.int64).reshape(-1, 3)
    out = np.zeros(cells.shape[0], dtype=np.float64)
    for i, (ix, iy, iz) in enumerate(cells):
        jx = ix + offsets[:, 0]
        jy = iy + offsets[:, 1]
        jz = iz + offsets[:, 2]
        if periodic:
            out[i] = F[np.mod(jz, nz), np.mod(jy, ny), np.mod(jx, nx)].sum()
        else:
            ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
            out[i] = F[jz[ok], jy[ok], jx[ok]].sum()
    return out


def pair_sums_fft(F: np.ndarray, offsets_list: Sequence[np.ndarray]) -> np.ndarray:
    """Order-2 sums sum_r F(r) W_s(r) = sum_{m in O_s} C(m) for every shell,
    C(m) = sum_r F(r) F(r + m) the circular autocorrelation of F, from one
    forward and one inverse library FFT (FP64).  On a periodic grid this is
    Eq. 12's numerator (or denominator); on a zero-outside grid it equals it
    when the guard band holds."""
    C = np.fft.irfftn(np.abs(np.fft.rfftn(F)) ** 2, s=F.shape, axes=(0, 1, 2))
    nz, ny, nx = F.shape
    out = np.zeros(len(offsets_list))
    for i, o in enumerate(offsets_list):
        out[i] = C[np.mod(o[:, 2], nz), np.mod(o[:, 1], ny), np.mod(o[:, 0], nx)].sum()
    return out


def guard_band_ok(fields: Iterable[np.ndarray], max_offset: Sequence[int]) -> bool:
    """Circular (FFT) convolution equals the zero-outside one at every cell
    where a field is non-zero iff, per axis, the periodic images cannot reach:
    (extent of the non-zero cells) + max|m| < n."""
    occ = None
    for F in fields:
        nz_ = F != 0
        occ = nz_ if occ is None else (occ | nz_)
    if occ is None or not occ.any():
        return True
    for axis, m in ((2, max_offset[0]), (1, max_offset[1]), (0, max_offset[2])):
        other = tuple(a for a in range(3) if a != axis)
        used = np.nonzero(occ.any(axis=other))[0]
        if int(used[-1] - used[0]) + int(m) >= occ.shape[axis]:
            return False
    return True


# ---------------------------------------------------------------------------
# Summation (Sec. 2.5, Eqs. 11-14)

def multisets(n_shells: int, k: int) -> List[Tuple[int, ...]]:
    """All s_1 <= ... <= s_k over range(n_shells), lexicographic order."""
    return list(itertools.combinations_with_replacement(range(n_shells), k))


def product_sums(W0: np.ndarray, W: Sequence[np.ndarray], order: int):
    """For every multiset of n - 1 = order - 1 shells: sum_r W0 prod W_{s_i}
    (Eq. 11's numerator, or its denominator when given B) and the sum of the
    absolute values of the same terms.  Returns (values, abs_values) in the
    order of ``multisets``."""
    sets = multisets(len(W), order - 1)
    vals = np.zeros(len(sets), dtype=np.float64)
    avals = np.zeros(len(sets), dtype=np.float64)
    for i, ms in enumerate(sets):
        t = W0.copy()
        for s in ms:
            t = t * W[s]
        vals[i] = t.sum()
        avals[i] = np.abs(t).sum()
    return vals, avals


def dense_tensor(values: np.ndarray, n_shells: int, k: int) -> np.ndarray:
    """Fill the symmetric [n_shells]^k tensor from per-multiset values."""
    T = np.zeros((n_shells,) * k, dtype=np.float64)
    for v, ms in zip(values, multisets(n_shells, k)):
        for p in set(itertools.permutations(ms)):
            T[p] = v
    return T


def xi_from(num: np.ndarray, den: np.ndarray) -> np.ndarray:
    """xi = num / den, NaN where den <= 0 (reading 7)."""
    num = np.asarray(num, np.float64)
    den = np.asarray(den, np.float64)
    out = np.full(num.shape, np.nan)
    ok = den > 0
    out[ok] = num[ok] / den[ok]
    return out


def xi_diagonal(W0, W1, B0, B1, order: int) -> float:
    """Equidistant n-point function (Eq. 14): sum W0 W1^(n-1) / sum B0 B1^(n-1)."""
    num = float(np.sum(W0 * W1 ** (order - 1)))
    den = float(np.sum(B0 * B1 ** (order - 1)))
    return num / den if den > 0 else float("nan")


def delta_field(D, R) -> np.ndarray:
    """Eq. 15 (reading 11): (D - R) / R where R > 0, else 0; FP64."""
    D = np.asarray(D, np.float64)
    R = np.asarray(R, np.float64)
    out = np.zeros(D.shape, np.float64)
    ok = R > 0
    out[ok] = (D[ok] - R[ok]) / R[ok]
    return out


def field_sums(grid, shells: Sequence[float], width: float, W0, F, orders: Sequence[int] = (2, 3),
               engine: str = "direct", rule: str = "center_bin") -> Dict[str, object]:
    """Eq. 16 for a continuous field (W0 = F = delta, reading 11) or a cross
    pair (W0 = Delta_0, F = Delta_1, reading 12): W_s = F *** K_s and per
    order n the sums over multisets of sum_r W0 prod W_{s_i} with the sums of
    their absolute terms."""
    W0 = np.asarray(W0, np.float64)
    F = np.asarray(F, np.float64)
    offs = [shell_offsets(s, width, grid.cell, rule) for s in shells]
    if engine == "direct":
        W = [convolve_direct(F, o, grid.periodic) for o in offs]
    elif engine == "fft":
        W = [convolve_fft(F, o) for o in offs]
    else:
        raise ValueError(engine)
    out: Dict[str, object] = dict(W=W, offsets=offs)
    for n in orders:
        v, a = product_sums(W0, W, n)
        out[f"num{n}"] = v
        out[f"abs_num{n}"] = a
        out[f"xi{n}"] = dense_tensor(v, len(shells), n - 1)
    return out


def product_map(W0, Ws, den2_s: float, n_box: int) -> np.ndarray:
    """Reading 13: W_0 W_s / <B_0 B_s> per cell, <B_0 B_s> = den_2(s) / N_box."""
    return np.asarray(W0, np.float64) * np.asarray(Ws, np.float64) / (den2_s / n_box)


def correlate(grid, shells: Sequence[float], width: float, data, randoms,
              orders: Sequence[int] = (2, 3), engine: str = "direct",
              rule: str = "center_bin", data_weights=None, random_weights=None,
              random_field=None, alpha: float = None, owned_z=None) -> Dict[str, object]:
    """The whole path for one catalog: mapping, convolution, summation.

    Returns a dict with D, R, dropped counts, alpha, N, Rt, the offset lists,
    W and B banks, and per order n: num, den, abs_num, abs_den (per multiset)
    and the dense xi tensor [N_s]^(n-1).  random_field, when given, is the
    randoms histogram itself (the factorised field of Eq. 7) and `randoms`
    is not read.

    One region of a catalog cut into slabs along z (reading 14): alpha, when
    given, replaces sum D / sum R (the whole catalog's ratio), and
    owned_z = (z0, z1) keeps the sums to the planes z0 <= z < z1 (W_0 = N
    and B_0 = Rt are zero elsewhere) while every plane of the grid, the halo
    included, enters the convolution.  The regions' num and den then add up
    to the whole catalog's (Eq. 19).
    """
    if data_weights is None:
        D, dropped_d = grid_counts(data.x, data.y, data.z, grid)
    else:  # weighted histograms (reading 8)
        D, _, dropped_d = grid_weights(data.x, data.y, data.z, data_weights, grid)
    if random_field is not None:
        R, dropped_r = np.asarray(random_field, np.float64), 0
    elif random_weights is None:
        R, dropped_r = grid_counts(randoms.x, randoms.y, randoms.z, grid)
    else:
        R, _, dropped_r = grid_weights(randoms.x, randoms.y, randoms.z, random_weights, grid)
    alpha, N, Rt = density_fields(D, R, alpha)
    offs = [shell_offsets(s, width, grid.cell, rule) for s in shells]
    if grid.periodic:
        for o in offs:
            if not check_periodic_support(o, grid.n):
                raise ValueError("shell support reaches half the periodic box")
    if engine == "direct":
        conv = lambda F, o: convolve_direct(F, o, grid.periodic)  # noqa: E731
    elif engine == "fft":
        if not grid.periodic:
            mmax = np.max([np.abs(o).max(axis=0) for o in offs if o.size], axis=0)
            if not guard_band_ok([D, R], mmax):
                raise ValueError("data reach the box faces: circular convolution differs")
        conv = convolve_fft
    else:
        raise ValueError(engine)
    W = [conv(N, o) for o in offs]
    B = [conv(Rt, o) for o in offs]
    out: Dict[str, object] = dict(D=D, R=R, dropped_d=dropped_d, dropped_r=dropped_r,
                                  alpha=alpha, N=N, Rt=Rt, offsets=offs, W=W, B=B)
    ns = len(shells)
    N0, Rt0 = N, Rt
    if owned_z is not None:
        z0, z1 = (int(v) for v in owned_z)
        keep = np.zeros(N.shape[0], dtype=bool)
        keep[z0:z1] = True
        N0 = np.where(keep[:, None, None], N, 0.0)
        Rt0 = np.where(keep[:, None, None], Rt, 0.0)
    for n in orders:
        num, anum = product_sums(N0, W, n)
        den, aden = product_sums(Rt0, B, n)
        out[f"num{n}"] = num
        out[f"den{n}"] = den
        out[f"abs_num{n}"] = anum
        out[f"abs_den{n}"] = aden
        out[f"xi{n}"] = dense_tensor(xi_from(num, den), ns, n - 1)
    return out
