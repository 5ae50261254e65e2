"""Checks that pin the FP64 oracle to facts fixed outside it.

Every check takes the oracle module as an argument and returns True when the
oracle agrees with the independent fact.  ``test_oracle_pins`` asserts each
one; ``test_oracle_mutations`` plants mistakes in the oracle and asserts that
at least one check then fails.

The independent facts used here:

* counts of points placed exactly at cell centres / edges (known by
  construction);
* lattice-point counts of a spherical shell, by brute-force enumeration in
  plain Python;
* ordered pair, triplet and higher counts of points at cell centres on a
  periodic grid, by brute force over the points with minimum-image integer
  separations: sum_r D W_{s_1} ... W_{s_k} equals the number of ordered
  tuples (i, j_1, .., j_k) with the separation i-j_t in shell s_t, and the
  same with signed weights for N = D - alpha R (Secs. 2.4-2.5, Eqs. 9-13);
* closed forms: a constant random field gives den = N_c c^n prod |O_s|;
  a delta field gives W_s = the indicator of the shell about the delta;
* the discrete Fourier transform written out as a cosine sum;
* invariances: shell relabelling, integer translations, linearity, region
  additivity (Eq. 19) and the equidistant diagonal (Eq. 14).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from synth import Catalog, GridSpec, lattice_catalog


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# independent helpers (no oracle code)

def brute_shell_count(radius, width, cell):
    """Number of integer vectors with (s - w/2) <= |m| g < (s + w/2)."""
    lo = max(radius - width / 2.0, 0.0)
    hi = radius + width / 2.0
    h = int(math.ceil(hi / cell)) + 1
    c = 0
    for i in range(-h, h + 1):
        for j in range(-h, h + 1):
            for k in range(-h, h + 1):
                d = math.sqrt(i * i + j * j + k * k) * cell
                if lo <= d < hi:
                    c += 1
    return c


def _in_shell(d2_cells, radius, width, cell):
    """Shell test on squared integer separations (cell units)."""
    lo = max(radius - width / 2.0, 0.0)
    hi = radius + width / 2.0
    d = np.sqrt(d2_cells.astype(np.float64)) * cell
    return (d >= lo) & (d < hi)


def _min_image(ci, cj, n):
    """Minimum-image integer separation cj - ci on a periodic axis of n."""
    d = np.mod(cj - ci, n)
    return np.where(d >= (n + 1) // 2, d - n, d)


def _sep2(cells_a, cells_b, n):
    d2 = np.zeros((cells_a.shape[0], cells_b.shape[0]), dtype=np.int64)
    for a in range(3):
        d = _min_image(cells_a[:, a][:, None], cells_b[:, a][None, :], n[a])
        d2 += d * d
    return d2


# ---------------------------------------------------------------------------
# mapping

def check_lattice_gridding(o) -> bool:
    """Cell-centred points on a non-cubic grid land in their own cells, and
    lower-edge points in the cell whose edge they sit on."""
    g = GridSpec((8, 6, 5), (-3.5, 2.0, 10.0), 2.5, False)
    rng = _rng(11)
    cells = np.stack([rng.integers(0, g.n[a], 60) for a in range(3)], axis=1)
    mult = rng.integers(1, 4, 60)
    expect = np.zeros((g.n[2], g.n[1], g.n[0]), dtype=np.int64)
    for (ix, iy, iz), m in zip(cells, mult):
        expect[iz, iy, ix] += m
    ok = True
    for where in ("centre", "edge"):
        cat = lattice_catalog(g, cells, mult, where=where)
        D, dropped = o.grid_counts(cat.x, cat.y, cat.z, g)
        ok &= dropped == 0 and D.shape == expect.shape and np.array_equal(D.astype(np.int64), expect)
    # just below a lower edge belongs to the previous cell
    e = np.float32(g.origin[0] + 3 * g.cell)
    below = np.nextafter(e, np.float32(-np.inf))
    cat = Catalog(np.array([e, below], np.float32), np.array([3.0, 3.0], np.float32),
                  np.array([11.0, 11.0], np.float32))
    D, _ = o.grid_counts(cat.x, cat.y, cat.z, g)
    ok &= int(D[0, 0, 3]) == 1 and int(D[0, 0, 2]) == 1
    return bool(ok)


def check_out_of_grid(o) -> bool:
    """Non-periodic: points outside [origin, origin + n g) are dropped and
    counted.  Periodic: x = L is cell 0 and x = -g/2 is cell n - 1."""
    g = GridSpec((4, 4, 4), (0.0, 0.0, 0.0), 1.0, False)
    x = np.array([-0.5, 4.0, 3.999, 0.0, 2.5], np.float32)
    y = np.array([1.5, 1.5, 1.5, 1.5, 9.0], np.float32)
    z = np.array([1.5, 1.5, 1.5, 1.5, 1.5], np.float32)
    D, dropped = o.grid_counts(x, y, z, g)
    ok = dropped == 3 and int(D.sum()) == 2 and int(D[1, 1, 3]) == 1 and int(D[1, 1, 0]) == 1
    gp = GridSpec((4, 4, 4), (0.0, 0.0, 0.0), 1.0, True)
    x = np.array([4.0, -0.5, 1.5], np.float32)
    D, dropped = o.grid_counts(x, np.full(3, 0.5, np.float32), np.full(3, 2.5, np.float32), gp)
    ok &= dropped == 0 and int(D[2, 0, 0]) == 1 and int(D[2, 0, 3]) == 1 and int(D[2, 0, 1]) == 1
    return bool(ok)


def check_alpha_and_fields(o) -> bool:
    """alpha = sum D / sum R; N = D - alpha R; Rt = alpha R (Eq. 8)."""
    D = np.array([[[3, 0], [1, 2]]], np.uint32)
    R = np.array([[[10, 4], [0, 6]]], np.uint32)
    alpha, N, Rt = o.density_fields(D, R)
    return bool(alpha == 0.3 and np.allclose(N, [[[0.0, -1.2], [1.0, 0.2]]], rtol=0, atol=1e-15)
                and np.allclose(Rt, [[[3.0, 1.2], [0.0, 1.8]]], rtol=0, atol=1e-15))


# ---------------------------------------------------------------------------
# kernels

SHELL_CASES = [(20.0, 10.0, 10.0), (40.0, 10.0, 10.0), (30.0, 8.0, 8.0), (34.0, 4.0, 8.0),
               (3.0, 1.0, 1.0), (2.0, 1.0, 1.0), (1.5, 1.0, 1.0), (50.0, 5.0, 5.0)]


def check_shell_counts(o) -> bool:
    """|O_s| equals a brute-force lattice count, the set is closed under sign
    flips and axis permutations, and every member obeys the shell bounds."""
    for s, w, g in SHELL_CASES:
        offs = o.shell_offsets(s, w, g)
        if offs.shape[0] != brute_shell_count(s, w, g):
            return False
        S = {tuple(int(v) for v in m) for m in offs}
        if len(S) != offs.shape[0]:
            return False
        for m in list(S)[:50]:
            for p in itertools.permutations(m):
                for sg in itertools.product((1, -1), repeat=3):
                    if tuple(a * b for a, b in zip(p, sg)) not in S:
                        return False
    return True


def check_intersect_rule(o) -> bool:
    """Rule "intersect": a cell is kept iff the sphere of radius s passes
    through the cell cube; checked against dense sampling of each cube."""
    s, g = 2.3, 1.0
    offs = o.shell_offsets(s, 0.0, g, rule="intersect")
    S = {tuple(int(v) for v in m) for m in offs}
    t = np.linspace(-0.5, 0.5, 41)
    px, py, pz = np.meshgrid(t, t, t, indexing="ij")
    for i in range(-4, 5):
        for j in range(-4, 5):
            for k in range(-4, 5):
                d = np.sqrt((i + px) ** 2 + (j + py) ** 2 + (k + pz) ** 2) * g
                lo, hi = d.min(), d.max()
                if abs(lo - s) < 0.03 or abs(hi - s) < 0.03:
                    continue  # too close to call by sampling
                if ((lo < s < hi) != ((i, j, k) in S)):
                    return False
    return True


def check_kernel_spectrum(o) -> bool:
    """The octant of K^/N_c equals the DFT written as a cosine sum over the
    offset list, divided by N_c; K^(0) N_c = |O_s|."""
    n = (10, 8, 6)
    offs = o.shell_offsets(2.0, 1.0, 1.0)
    Kh = o.kernel_spectrum_octant(offs, n)
    Nc = n[0] * n[1] * n[2]
    if Kh.shape != (n[2] // 2 + 1, n[1] // 2 + 1, n[0] // 2 + 1):
        return False
    if abs(Kh[0, 0, 0] * Nc - offs.shape[0]) > 1e-9:
        return False
    for kz in range(n[2] // 2 + 1):
        for ky in range(n[1] // 2 + 1):
            for kx in range(n[0] // 2 + 1):
                ph = 2 * math.pi * (kx * offs[:, 0] / n[0] + ky * offs[:, 1] / n[1] + kz * offs[:, 2] / n[2])
                if abs(np.cos(ph).sum() / Nc - Kh[kz, ky, kx]) > 1e-12:
                    return False
    return True


# ---------------------------------------------------------------------------
# convolution + summation: exact counting identities

def _centre_points(grid, count, seed):
    rng = _rng(seed)
    cells = np.stack([rng.integers(0, grid.n[a], count) for a in range(3)], axis=1)
    return cells, lattice_catalog(grid, cells)


PGRID = GridSpec((9, 8, 7), (0.0, 0.0, 0.0), 2.0, True)
PSHELLS = [(2.5, 1.0), (3.6, 1.2), (5.0, 2.0)]


def _cell_rule_ok(o, shells, grid):
    return all(o.check_periodic_support(o.shell_offsets(s, w, grid.cell), grid.n) for s, w in shells)


def check_pair_counts(o) -> bool:
    """sum_r D W_s = #ordered pairs (i, j) with separation in shell s."""
    g = PGRID
    if not _cell_rule_ok(o, PSHELLS, g):
        return False
    cells, cat = _centre_points(g, 45, 5)
    D, _ = o.grid_counts(cat.x, cat.y, cat.z, g)
    Dd = D.astype(np.float64)
    d2 = _sep2(cells, cells, g.n)
    for s, w in PSHELLS:
        W = o.convolve_direct(Dd, o.shell_offsets(s, w, g.cell), True)
        got = float((Dd * W).sum())
        want = int(_in_shell(d2, s, w, g.cell).sum())
        if got != want:
            return False
    return True


def check_triplet_counts(o) -> bool:
    """sum_r D W_a W_b = #ordered (i, j, k), sep(i,j) in a, sep(i,k) in b,
    j = k allowed (Eq. 13's numerator on cell-centred points)."""
    g = PGRID
    cells, cat = _centre_points(g, 30, 6)
    D, _ = o.grid_counts(cat.x, cat.y, cat.z, g)
    Dd = D.astype(np.float64)
    d2 = _sep2(cells, cells, g.n)
    for (sa, wa), (sb, wb) in [(PSHELLS[0], PSHELLS[1]), (PSHELLS[1], PSHELLS[1]), (PSHELLS[2], PSHELLS[0])]:
        Wa = o.convolve_direct(Dd, o.shell_offsets(sa, wa, g.cell), True)
        Wb = o.convolve_direct(Dd, o.shell_offsets(sb, wb, g.cell), True)
        got = float((Dd * Wa * Wb).sum())
        A = _in_shell(d2, sa, wa, g.cell)
        B = _in_shell(d2, sb, wb, g.cell)
        want = int(np.einsum("ij,ik->", A.astype(np.int64), B.astype(np.int64)))
        if got != want:
            return False
    return True


def check_product_sums_high_order(o) -> bool:
    """product_sums for n = 2..5 on cell-centred points equals
    sum_i prod_t cnt_{s_t}(i), cnt_s(i) = #j with sep(i, j) in s."""
    g = PGRID
    cells, cat = _centre_points(g, 25, 7)
    D, _ = o.grid_counts(cat.x, cat.y, cat.z, g)
    Dd = D.astype(np.float64)
    d2 = _sep2(cells, cells, g.n)
    W = [o.convolve_direct(Dd, o.shell_offsets(s, w, g.cell), True) for s, w in PSHELLS]
    cnt = [_in_shell(d2, s, w, g.cell).sum(axis=1).astype(np.int64) for s, w in PSHELLS]
    for order in (2, 3, 4, 5):
        vals, avals = o.product_sums(Dd, W, order)
        sets = list(itertools.combinations_with_replacement(range(len(PSHELLS)), order - 1))
        if len(vals) != len(sets):
            return False
        for v, av, ms in zip(vals, avals, sets):
            want = int(np.prod(np.stack([cnt[s] for s in ms]), axis=0).sum())
            if v != want or av != want:
                return False
    return True


def check_signed_pairs(o) -> bool:
    """With N = D - alpha R built from data (+1) and randoms (-alpha) at cell
    centres: sum_r N W_s = sum_{i,j} w_i w_j [sep(i,j) in s], and likewise
    sum_r Rt B_s over the randoms alone with weight alpha."""
    g = PGRID
    cd, dat = _centre_points(g, 20, 8)
    cr, ran = _centre_points(g, 70, 9)
    D, _ = o.grid_counts(dat.x, dat.y, dat.z, g)
    R, _ = o.grid_counts(ran.x, ran.y, ran.z, g)
    alpha, N, Rt = o.density_fields(D, R)
    if abs(alpha - 20.0 / 70.0) > 1e-15:
        return False
    cells = np.concatenate([cd, cr])
    wts = np.concatenate([np.ones(20), -alpha * np.ones(70)])
    d2 = _sep2(cells, cells, g.n)
    d2r = _sep2(cr, cr, g.n)
    for s, w in PSHELLS:
        offs = o.shell_offsets(s, w, g.cell)
        W = o.convolve_direct(N, offs, True)
        B = o.convolve_direct(Rt, offs, True)
        want = float(wts @ (_in_shell(d2, s, w, g.cell) @ wts))
        wantr = alpha * alpha * float(_in_shell(d2r, s, w, g.cell).sum())
        if abs((N * W).sum() - want) > 1e-10 * max(1.0, abs(want)):
            return False
        if abs((Rt * B).sum() - wantr) > 1e-10 * max(1.0, abs(wantr)):
            return False
    return True


def check_delta_response(o) -> bool:
    """A single unit cell c gives W_s(r) = 1 exactly where c - r is in O_s
    (periodic and zero-outside boundaries)."""
    for periodic in (True, False):
        n = (9, 8, 7)
        F = np.zeros((n[2], n[1], n[0]))
        c = (4, 3, 3)
        F[c[2], c[1], c[0]] = 1.0
        offs = o.shell_offsets(2.5, 1.0, 1.0)
        W = o.convolve_direct(F, offs, periodic)
        want = np.zeros_like(F)
        for mx, my, mz in offs:
            rx, ry, rz = c[0] - mx, c[1] - my, c[2] - mz
            if periodic:
                want[rz % n[2], ry % n[1], rx % n[0]] += 1
            elif 0 <= rx < n[0] and 0 <= ry < n[1] and 0 <= rz < n[2]:
                want[rz, ry, rx] += 1
        if not np.array_equal(W, want):
            return False
    return True


def check_fft_engine(o) -> bool:
    """The FFT engine equals the direct engine on a periodic grid."""
    rng = _rng(12)
    F = rng.normal(size=(7, 8, 9))
    for s, w in PSHELLS:
        offs = o.shell_offsets(s, w, 2.0)
        a = o.convolve_direct(F, offs, True)
        b = o.convolve_fft(F, offs)
        if np.abs(a - b).max() > 1e-12 * max(1.0, np.abs(a).max()):
            return False
    return True


def _uniform_lattice_case(o, c_per_cell=1):
    g = GridSpec((10, 9, 8), (0.0, 0.0, 0.0), 1.0, True)
    allc = np.stack(np.meshgrid(np.arange(10), np.arange(9), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    rng = _rng(13)
    dat = lattice_catalog(g, allc[rng.integers(0, allc.shape[0], 50)])
    ran = lattice_catalog(g, allc, np.full(allc.shape[0], c_per_cell))
    return g, dat, ran


def check_constant_field_den(o) -> bool:
    """Randoms filling every cell equally (R = 2) give Rt = c = 2 alpha
    everywhere and den_n = N_c c^n prod |O_s| (closed form)."""
    g, dat, ran = _uniform_lattice_case(o, 2)
    shells = (1.5, 2.5, 3.2)
    res = o.correlate(g, shells, 1.0, dat, ran, orders=(2, 3, 4, 5))
    alpha = 50.0 / (2 * g.n_cells)
    c = 2 * alpha  # Rt = alpha R with R = 2 in every cell
    sizes = [brute_shell_count(s, 1.0, 1.0) for s in shells]
    for n in (2, 3, 4, 5):
        sets = list(itertools.combinations_with_replacement(range(3), n - 1))
        for v, ms in zip(res[f"den{n}"], sets):
            want = g.n_cells * c ** n * np.prod([sizes[s] for s in ms])
            if abs(v - want) > 1e-10 * want:
                return False
    return True


def _clustered_case(seed=21):
    from synth import neyman_scott_box, uniform_box
    g = GridSpec((12, 10, 8), (0.0, 0.0, 0.0), 10.0, True)
    dat = neyman_scott_box(seed, 30, 8, 6.0, 80.0)
    # clip into the non-cubic box (x < 120, y < 100, z < 80)
    dat = Catalog(np.mod(dat.x * 1.5, 120.0), np.mod(dat.y * 1.25, 100.0), dat.z)
    ran = uniform_box(seed + 1, 2000, 80.0)
    ran = Catalog(np.mod(ran.x * 1.5, 120.0), np.mod(ran.y * 1.25, 100.0), ran.z)
    return g, dat, ran


CSHELLS = (15.0, 25.0, 32.0)


def check_relabel_shells(o) -> bool:
    """Passing the shells in another order permutes the xi tensors the same
    way (no mix-up between shell labels and W banks)."""
    g, dat, ran = _clustered_case()
    a = o.correlate(g, CSHELLS, 10.0, dat, ran, orders=(2, 3, 4))
    perm = (2, 0, 1)
    b = o.correlate(g, tuple(CSHELLS[p] for p in perm), 10.0, dat, ran, orders=(2, 3, 4))
    for n in (2, 3, 4):
        A = a[f"xi{n}"]
        B = b[f"xi{n}"]
        idx = np.ix_(*([list(perm)] * (n - 1)))
        if not np.allclose(A[idx], B, rtol=1e-12, atol=0, equal_nan=True):
            return False
        if not np.allclose(A, np.swapaxes(A, 0, -1), rtol=1e-12, equal_nan=True):
            return False
    return True


def check_translation(o) -> bool:
    """Moving every point by whole cells on a periodic grid leaves num, den
    and xi unchanged."""
    g, dat, ran = _clustered_case()
    a = o.correlate(g, CSHELLS, 10.0, dat, ran, orders=(2, 3))
    sh = (30.0, 70.0, 10.0)

    def mv(c):
        return Catalog(np.mod(c.x.astype(np.float64) + sh[0], 120.0),
                       np.mod(c.y.astype(np.float64) + sh[1], 100.0),
                       np.mod(c.z.astype(np.float64) + sh[2], 80.0))
    b = o.correlate(g, CSHELLS, 10.0, mv(dat), mv(ran), orders=(2, 3))
    for n in (2, 3):
        for key in ("num", "den"):
            x, y = a[f"{key}{n}"], b[f"{key}{n}"]
            if np.abs(x - y).max() > 1e-9 * np.abs(x).max():
                return False
    return True


def check_linearity(o) -> bool:
    """W of N = D - alpha R equals W(D) - alpha W(R) (Eq. 9 is linear)."""
    g, dat, ran = _clustered_case()
    D, _ = o.grid_counts(dat.x, dat.y, dat.z, g)
    R, _ = o.grid_counts(ran.x, ran.y, ran.z, g)
    alpha, N, _ = o.density_fields(D, R)
    offs = o.shell_offsets(25.0, 10.0, 10.0)
    a = o.convolve_direct(N, offs, True)
    b = o.convolve_direct(D.astype(np.float64), offs, True) - alpha * o.convolve_direct(R.astype(np.float64), offs, True)
    return bool(np.abs(a - b).max() <= 1e-12 * np.abs(b).max())


def check_region_additivity(o) -> bool:
    """Two regions further apart than the largest shell, each with its own
    alpha, in one zero-outside box: the product sums of the combined field
    are the sums over the regions (Eq. 19)."""
    g = GridSpec((24, 10, 10), (0.0, 0.0, 0.0), 1.0, False)
    rng = _rng(31)

    def region(x0, nd, nr):
        cd = np.stack([rng.integers(x0, x0 + 6, nd), rng.integers(2, 8, nd), rng.integers(2, 8, nd)], 1)
        cr = np.stack([rng.integers(x0, x0 + 6, nr), rng.integers(2, 8, nr), rng.integers(2, 8, nr)], 1)
        D, _ = o.grid_counts(*_xyz(lattice_catalog(g, cd)), g)
        R, _ = o.grid_counts(*_xyz(lattice_catalog(g, cr)), g)
        return o.density_fields(D, R)

    aA, NA, RA = region(1, 40, 200)
    aB, NB, RB = region(16, 25, 300)
    shells = [(1.5, 1.0), (2.5, 1.0), (3.5, 1.0)]
    offs = [o.shell_offsets(s, w, 1.0) for s, w in shells]

    def sums(N, Rt):
        W = [o.convolve_direct(N, x, False) for x in offs]
        B = [o.convolve_direct(Rt, x, False) for x in offs]
        return o.product_sums(N, W, 3)[0], o.product_sums(Rt, B, 3)[0]
    nA, dA = sums(NA, RA)
    nB, dB = sums(NB, RB)
    nC, dC = sums(NA + NB, RA + RB)
    return bool(np.allclose(nC, nA + nB, rtol=1e-12, atol=1e-9) and np.allclose(dC, dA + dB, rtol=1e-12))


def _xyz(c):
    return c.x, c.y, c.z


def check_diagonal(o) -> bool:
    """xi_n(s, .., s) equals Eq. 14 evaluated on its own."""
    g, dat, ran = _clustered_case()
    res = o.correlate(g, CSHELLS, 10.0, dat, ran, orders=(2, 3, 4, 5))
    for n in (2, 3, 4, 5):
        T = res[f"xi{n}"]
        for s in range(len(CSHELLS)):
            want = o.xi_diagonal(res["N"], res["W"][s], res["Rt"], res["B"][s], n)
            if not math.isclose(T[(s,) * (n - 1)], want, rel_tol=1e-12):
                return False
    return True


def check_sum_of_w(o) -> bool:
    """On a periodic grid sum_r W_s = (sum_r N) |O_s|."""
    rng = _rng(41)
    F = rng.normal(size=(8, 9, 10))
    for s, w in PSHELLS:
        offs = o.shell_offsets(s, w, 2.0)
        W = o.convolve_direct(F, offs, True)
        if abs(W.sum() - F.sum() * offs.shape[0]) > 1e-10 * np.abs(F).sum() * offs.shape[0]:
            return False
    return True


def check_sampled_cells(o) -> bool:
    """w_at_cells agrees with the full convolution at sampled cells."""
    rng = _rng(42)
    F = rng.normal(size=(7, 8, 9))
    offs = o.shell_offsets(3.6, 1.2, 2.0)
    cells = np.stack([rng.integers(0, 9, 20), rng.integers(0, 8, 20), rng.integers(0, 7, 20)], 1)
    for periodic in (True, False):
        W = o.convolve_direct(F, offs, periodic)
        got = o.w_at_cells(F, offs, cells, periodic)
        if np.abs(got - W[cells[:, 2], cells[:, 1], cells[:, 0]]).max() > 1e-12:
            return False
    return True


def check_multisets(o) -> bool:
    """C(N_s + k - 1, k) sorted multisets in lexicographic order."""
    for ns in (1, 4, 16):
        for k in (1, 2, 3, 4):
            m = o.multisets(ns, k)
            if len(m) != math.comb(ns + k - 1, k) or m != sorted(m):
                return False
            if any(list(t) != sorted(t) for t in m):
                return False
    return True


def check_guard_band(o) -> bool:
    """The guard-band test accepts exactly when periodic images cannot reach:
    on a non-periodic grid with data inside the band, FFT and direct agree."""
    F = np.zeros((16, 16, 16))
    F[5:11, 6:9, 4:12] = 1.0
    offs = o.shell_offsets(3.0, 1.0, 1.0)
    m = np.abs(offs).max(axis=0)
    if not o.guard_band_ok([F], m):
        return False
    a = o.convolve_direct(F, offs, False)
    b = o.convolve_fft(F, offs)
    ok = np.abs((a - b) * (F != 0)).max() < 1e-12
    G = np.zeros((16, 16, 16))
    G[0, 0, 0] = 1.0
    G[0, 0, 14] = 1.0
    return bool(ok and not o.guard_band_ok([G], m))


def check_pair_sums_fft(o) -> bool:
    """The autocorrelation route to the order-2 sums equals the brute-force
    ordered pair counts of cell-centred points."""
    g = PGRID
    cells, cat = _centre_points(g, 45, 5)
    D, _ = o.grid_counts(cat.x, cat.y, cat.z, g)
    d2 = _sep2(cells, cells, g.n)
    got = o.pair_sums_fft(D.astype(np.float64), [o.shell_offsets(s, w, g.cell) for s, w in PSHELLS])
    want = [int(_in_shell(d2, s, w, g.cell).sum()) for s, w in PSHELLS]
    return bool(np.allclose(got, want, rtol=0, atol=1e-6))


def check_grid_weights(o) -> bool:
    """Weighted histograms (reading 8) against facts outside the function:
    unit weights give the counts; small integer weights give the weighted
    counts (exact); random weights differ from an FP64 sum by at most
    2^-33 per point; exact rational arithmetic on a tiny case (signed
    weights, ties of the rounding); non-finite weights are dropped."""
    from fractions import Fraction
    g = GridSpec((6, 5, 4), (1.0, -2.0, 0.5), 1.5, False)
    rng = _rng(41)
    cells = np.stack([rng.integers(-1, g.n[a] + 1, 400) for a in range(3)], axis=1)
    cat = lattice_catalog(g, cells)
    D, dropped = o.grid_counts(cat.x, cat.y, cat.z, g)
    Dw, tot, dw = o.grid_weights(cat.x, cat.y, cat.z, np.ones(400, np.float32), g)
    ok = dw == dropped and np.array_equal(Dw, D.astype(np.float64)) and tot == float(D.sum())
    k = rng.integers(1, 4, 400).astype(np.float32)
    Dk, _, _ = o.grid_weights(cat.x, cat.y, cat.z, k, g)
    expect = np.zeros(D.shape, np.float64)
    for (ix, iy, iz), kv in zip(cells, k):
        if 0 <= ix < g.n[0] and 0 <= iy < g.n[1] and 0 <= iz < g.n[2]:
            expect[iz, iy, ix] += float(kv)
    ok &= np.array_equal(Dk, expect)
    w = rng.uniform(0.1, 2.0, 400).astype(np.float32)
    Dr, _, _ = o.grid_weights(cat.x, cat.y, cat.z, w, g)
    fp = np.zeros(D.shape, np.float64)
    for (ix, iy, iz), wv in zip(cells, w):
        if 0 <= ix < g.n[0] and 0 <= iy < g.n[1] and 0 <= iz < g.n[2]:
            fp[iz, iy, ix] += float(wv)
    ok &= bool(np.all(np.abs(Dr - fp) <= D.astype(np.float64) * 2.0 ** -33 + 1e-15))
    # tiny exact case: three points in one cell, signed weights, a rounding tie
    tie = np.float32(3.0 * 2.0 ** -33)           # 1.5 units of 2^-32: rounds to 2 (even)
    wt = np.array([0.75, -0.25, tie], np.float32)
    one = lattice_catalog(g, np.array([[2, 1, 3]] * 3))
    Dt, tt, _ = o.grid_weights(one.x, one.y, one.z, wt, g)
    want = Fraction(3, 4) - Fraction(1, 4) + Fraction(2, 2 ** 32)
    ok &= Fraction(float(Dt[3, 1, 2])) == want and Fraction(tt) == want and float(Dt.sum()) == float(want)
    # non-finite weights are dropped
    wn = np.array([1.0, np.nan, np.inf], np.float32)
    Dn, _, dn = o.grid_weights(one.x, one.y, one.z, wn, g)
    ok &= dn == 2 and float(Dn.sum()) == 1.0
    return bool(ok)


def check_sky_coordinates(o) -> bool:
    """r(z) of Eq. 3 against closed forms: Einstein-de Sitter (O_M = 1:
    2 (c/H0) (1 - 1/sqrt(1+z))), pure Lambda (O_L = 1: c z / H0), curvature
    only (O_k = 1: (c/H0) ln(1+z)); Eqs. 4-6 on the axes and |X| = r."""
    z = np.array([0.0, 0.05, 0.3, 0.57, 1.0, 2.5])
    c, h0 = 299792.458, 67.7
    ok = np.allclose(o.comoving_distance(z, h0, 1.0, 0.0, 0.0, c),
                     2.0 * c / h0 * (1.0 - 1.0 / np.sqrt(1.0 + z)), rtol=1e-12, atol=1e-9)
    ok &= np.allclose(o.comoving_distance(z, h0, 0.0, 0.0, 1.0, c), c * z / h0, rtol=1e-12, atol=1e-9)
    ok &= np.allclose(o.comoving_distance(z, h0, 0.0, 1.0, 0.0, c), c / h0 * np.log1p(z), rtol=1e-12, atol=1e-9)
    # a flat LCDM distance grows with z and lies between the EdS and Lambda ones
    rl = o.comoving_distance(z, 100.0, 0.307, 0.0, 0.693, 300000.0)
    ok &= bool(np.all(np.diff(rl) > 0))
    ok &= bool(np.all(rl[1:] < 300000.0 / 100.0 * z[1:]))
    ok &= bool(np.all(rl[1:] > 2 * 3000.0 * (1 - 1 / np.sqrt(1 + z[1:]))))
    ra = np.array([0.0, 90.0, 0.0, 180.0, 33.0])
    dec = np.array([0.0, 0.0, 90.0, 0.0, -41.0])
    zz = np.full(5, 0.5)
    X, Y, Z = o.sky_to_cartesian(ra, dec, zz, 100.0, 0.307, 0.0, 0.693, 300000.0)
    r = o.comoving_distance(zz, 100.0, 0.307, 0.0, 0.693, 300000.0)
    ok &= np.allclose([X[0], Y[0], Z[0]], [r[0], 0, 0], atol=1e-9)
    ok &= np.allclose([X[1], Y[1], Z[1]], [0, r[1], 0], atol=1e-9)
    ok &= np.allclose([X[2], Y[2], Z[2]], [0, 0, r[2]], atol=1e-9)
    ok &= np.allclose([X[3], Y[3], Z[3]], [-r[3], 0, 0], atol=1e-9)
    ok &= np.allclose(np.sqrt(X ** 2 + Y ** 2 + Z ** 2), r, rtol=1e-14)
    ok &= bool(Z[4] < 0 and X[4] > 0 and Y[4] > 0)
    return bool(ok)



def _sel(**kw):
    base = dict(n_tot=1.0e5, p_ang=np.full((1, 1), 1.0 / (4.0 * np.pi)), p_z=np.array([1.0 / 0.04]),
                z_lo=0.02, z_hi=0.06, z_max=0.065, h0=100.0, omega_m=0.0, omega_k=0.0, omega_l=1.0,
                c=300000.0)
    base.update(kw)
    return base


def check_factorised_randoms(o) -> bool:
    """Eq. 7 (reading 10) against facts outside the function: P_ang (per
    steradian) and P_z (per unit z) are probability densities, so the field
    sums to N_tot over a grid that covers the shell (within the cells'
    discretisation, 4 % on 20-unit cells), with masks in right ascension, declination and
    redshift that leave nothing on the masked side; in an Einstein-de Sitter
    universe, where 1 + z = (1 - r H0 / 2c)^-2 and dz/dr = (H0/c)(1+z)^1.5,
    each cell's value follows in closed form; cells beyond r(z_max) are 0."""
    g = GridSpec((20, 20, 20), (-200.0, -200.0, -200.0), 20.0, False)
    nx, ny, nz = g.n
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = g.origin[0] + (ix + 0.5) * g.cell
    Y = g.origin[1] + (iy + 0.5) * g.cell
    Z = g.origin[2] + (iz + 0.5) * g.cell
    # pure Lambda: r = c z / H0 over [60, 180] h^-1 Mpc, uniform densities
    R = o.factorised_randoms(g, **_sel())
    ok = abs(R.sum() / 1.0e5 - 1.0) < 0.04 and float(R[np.sqrt(X * X + Y * Y + Z * Z) > 195.0].max()) == 0.0
    # northern sky only: P_ang = 1 / (2 pi) for dec >= 0
    R = o.factorised_randoms(g, **_sel(p_ang=np.array([[0.0], [1.0 / (2.0 * np.pi)]])))
    ok &= abs(R.sum() / 1.0e5 - 1.0) < 0.04 and float(R[Z < 0].max()) == 0.0
    # one quadrant in right ascension, 90 <= ra < 180 (X < 0 < Y): P_ang = 1 / pi
    pa = np.zeros((1, 4))
    pa[0, 1] = 1.0 / np.pi
    R = o.factorised_randoms(g, **_sel(p_ang=pa))
    ok &= abs(R.sum() / 1.0e5 - 1.0) < 0.04 and float(R[~((X < 0) & (Y > 0))].max()) == 0.0
    # the far half of the redshift range: nothing below r = 120
    R = o.factorised_randoms(g, **_sel(p_z=np.array([0.0, 2.0 / 0.04])))
    r = np.sqrt(X * X + Y * Y + Z * Z)
    ok &= abs(R.sum() / 1.0e5 - 1.0) < 0.04 and float(R[r < 119.0].max()) == 0.0
    # Einstein-de Sitter closed form at sampled cells, a non-uniform sky
    rng = _rng(57)
    pa = rng.uniform(0.5, 1.5, (6, 12))
    pz = rng.uniform(0.5, 1.5, 5)
    sel = _sel(p_ang=pa, p_z=pz, omega_m=1.0, omega_l=0.0, h0=70.0, c=299792.458, z_lo=0.02, z_hi=0.08,
               z_max=0.09)
    cells = np.stack([rng.integers(0, 20, 60) for _ in range(3)], axis=1)
    got = o.factorised_randoms_at(cells, g, **sel)
    ctr = np.asarray(g.origin) + (cells + 0.5) * g.cell
    rr = np.sqrt((ctr * ctr).sum(axis=1))
    zz = (1.0 - rr * 70.0 / (2.0 * 299792.458)) ** -2.0 - 1.0
    ra = np.degrees(np.arctan2(ctr[:, 1], ctr[:, 0])) % 360.0
    dec = np.degrees(np.arcsin(ctr[:, 2] / rr))
    want = np.zeros(len(cells))
    live = (zz >= 0.02) & (zz < 0.08)
    for i in np.nonzero(live)[0]:
        pav = pa[int((dec[i] + 90.0) // 30.0), int(ra[i] // 30.0)]
        pzv = pz[int((zz[i] - 0.02) // 0.012)]
        want[i] = 1.0e5 * pav * pzv * (70.0 / 299792.458) * (1.0 + zz[i]) ** 1.5 * 8000.0 / rr[i] ** 2
    ok &= bool(live.sum() > 10) and bool(np.allclose(got, want, rtol=1e-9, atol=0.0))
    return bool(ok)



def check_delta_field(o) -> bool:
    """Eq. 15 (reading 11) by hand and by its special cases: D = R gives 0,
    D = 2R gives 1, cells with R = 0 give 0 whatever D holds."""
    ok = np.allclose(o.delta_field(np.array([3.0, 1.0, 5.0]), np.array([2.0, 0.0, 4.0])), [0.5, 0.0, 0.25],
                     rtol=0, atol=1e-15)
    rng = _rng(61)
    R = rng.uniform(0.5, 2.0, (6, 5, 4))
    R[0, 0, :] = 0.0
    D = rng.uniform(0.0, 3.0, R.shape)
    ok &= float(np.abs(o.delta_field(R, R)).max()) == 0.0
    two = o.delta_field(2.0 * R, R)
    ok &= bool(np.all(two[R > 0] == 1.0)) and bool(np.all(two[R == 0] == 0.0))
    ok &= bool(np.all(o.delta_field(D, R)[0, 0, :] == 0.0))
    return bool(ok)


def check_field_sums(o) -> bool:
    """Eq. 16 for continuous and cross fields (readings 11, 12): a constant
    field c on a periodic grid gives N_c c^n prod |O_s| (brute-force shell
    sizes); point fields give brute-force pair and triplet sums (W_0 = u at
    cell a, the convolved field v_b at cells b: num_2(s) = u sum_{b in s} v_b,
    num_3(s, t) = u (sum_{b in s} v_b)(sum_{b in t} v_b)); the cross sum of
    order 2 is symmetric in its two fields (K_s is even)."""
    g = GridSpec((12, 12, 12), (0.0, 0.0, 0.0), 1.0, True)
    shells, width = (1.5, 2.5, 3.4), 1.0
    c = 0.7
    F = np.full((12, 12, 12), c)
    res = o.field_sums(g, shells, width, F, F, orders=(2, 3))
    sizes = [brute_shell_count(s, width, 1.0) for s in shells]
    ok = True
    for n in (2, 3):
        for v, ms in zip(res[f"num{n}"], itertools.combinations_with_replacement(range(3), n - 1)):
            want = g.n_cells * c ** n * np.prod([sizes[s] for s in ms])
            ok &= abs(v - want) <= 1e-10 * want
    # point fields: W_0 at one cell, the convolved field at ten others
    rng = _rng(62)
    a = np.array([[5, 6, 4]])
    bs = np.unique(np.stack([rng.integers(2, 10, 10) for _ in range(3)], axis=1), axis=0)
    bs = bs[np.any(bs != a[0], axis=1)]
    W0 = np.zeros((12, 12, 12))
    W0[a[0, 2], a[0, 1], a[0, 0]] = 1.3
    F = np.zeros((12, 12, 12))
    v = rng.uniform(-1.0, 2.0, len(bs))
    for (x, y, z), vb in zip(bs, v):
        F[z, y, x] = vb
    res = o.field_sums(g, shells, width, W0, F, orders=(2, 3))
    d2 = _sep2(a, bs, g.n)[0]
    per = [float(np.sum(v[_in_shell(d2, s, width, 1.0)])) for s in shells]
    ok &= np.allclose(res["num2"], [1.3 * per[s] for s in range(3)], rtol=1e-12, atol=1e-12)
    want3 = [1.3 * per[s] * per[t] for s, t in itertools.combinations_with_replacement(range(3), 2)]
    ok &= np.allclose(res["num3"], want3, rtol=1e-12, atol=1e-12)
    ok &= bool(any(abs(x) > 0.1 for x in res["num2"]))
    # symmetry of the order-2 cross sum on a non-periodic grid
    gb = GridSpec((9, 8, 7), (0.0, 0.0, 0.0), 1.0, False)
    f0 = rng.normal(size=(7, 8, 9))
    f1 = rng.normal(size=(7, 8, 9))
    x01 = o.field_sums(gb, shells, width, f0, f1, orders=(2,))["num2"]
    x10 = o.field_sums(gb, shells, width, f1, f0, orders=(2,))["num2"]
    ok &= np.allclose(x01, x10, rtol=1e-12, atol=1e-12) and not np.allclose(x01, o.field_sums(
        gb, shells, width, f0, f0, orders=(2,))["num2"])
    return bool(ok)


def check_product_map(o) -> bool:
    """Reading 13 against the sums: the map times <B_0 B_s> summed over the
    cells is num_2(s); with Rt and N constant the map is the same in every
    cell, c_N^2 |O_s| / (c_R^2 |O_s|) = (c_N / c_R)^2."""
    g, dat, ran = _clustered_case()
    res = o.correlate(g, CSHELLS, 10.0, dat, ran, orders=(2,))
    ok = True
    for s in range(len(CSHELLS)):
        m = o.product_map(res["N"], res["W"][s], float(res["den2"][s]), g.n_cells)
        ok &= abs(float(m.sum()) * float(res["den2"][s]) / g.n_cells - float(res["num2"][s])) <= 1e-9 * (
            abs(float(res["abs_num2"][s])) + 1e-30)
    # constant fields: N = 0.3, Rt = 1.2 everywhere, |O_s| offsets
    gc = GridSpec((10, 10, 10), (0.0, 0.0, 0.0), 1.0, True)
    size = brute_shell_count(2.5, 1.0, 1.0)
    den2 = gc.n_cells * 1.2 * 1.2 * size
    m = o.product_map(np.full((10, 10, 10), 0.3), np.full((10, 10, 10), 0.3 * size), den2, gc.n_cells)
    ok &= np.allclose(m, (0.3 / 1.2) ** 2, rtol=1e-12)
    return bool(ok)


# ---------------------------------------------------------------------------
# boundary support and the xi rule (readings 4 and 7)

def _wraps_distinct(offsets, n):
    """Brute force: do the offsets stay pairwise distinct once every axis is
    taken mod n?"""
    seen = set()
    for m in offsets:
        key = tuple(int(m[a]) % int(n[a]) for a in range(3))
        if key in seen:
            return False
        seen.add(key)
    return True


def check_periodic_support(o) -> bool:
    """On each axis separately, offsets filling -m..m stay distinct after
    wrapping exactly when 2m < n; the oracle's support test must give the
    brute-force answer at n = 2m - 1, 2m, 2m + 1, with the other two axes
    long enough not to matter (and of different lengths, so that an axis
    mix-up shows)."""
    for m in (2, 3, 5):
        line = np.arange(-m, m + 1, dtype=np.int64)
        for a in range(3):
            off = np.zeros((line.size, 3), dtype=np.int64)
            off[:, a] = line
            # a second, shorter line on the next axis keeps the set 3D
            short = np.zeros((3, 3), dtype=np.int64)
            short[:, (a + 1) % 3] = (-1, 0, 1)
            off = np.concatenate([off, short[[0, 2]]])
            for n_a in (2 * m - 1, 2 * m, 2 * m + 1):
                n = [4 * m + 3 + 2 * b for b in range(3)]
                n[a] = n_a
                want = _wraps_distinct(off, n)
                if want != (2 * m < n_a):
                    return False
                if bool(o.check_periodic_support(off, n)) != want:
                    return False
    return True


def check_xi_nonpositive_den(o) -> bool:
    """Reading 7: xi = num / den where den > 0 and NaN where den <= 0, both
    on given arrays and end to end: randoms in a single cell give B_s = 0 at
    that cell for a shell that excludes the zero offset, so every den is
    exactly 0 and every xi NaN, while the data's num stay finite."""
    num = np.array([1.0, 2.0, -3.0, 4.0, 5.0])
    den = np.array([2.0, 0.0, -1.0, 8.0, -0.0])
    xi = o.xi_from(num, den)
    if not (xi[0] == 0.5 and xi[3] == 0.5 and np.isnan(xi[1]) and np.isnan(xi[2]) and np.isnan(xi[4])):
        return False
    g = GridSpec((8, 8, 8), (0.0, 0.0, 0.0), 1.0, True)
    one = lattice_catalog(g, np.array([[3, 4, 5]] * 4))
    cells, data = _centre_points(g, 30, 17)
    r = o.correlate(g, (2.0, 3.0), 1.0, data, one, orders=(2, 3), engine="direct")
    for n in (2, 3):
        if not np.all(r[f"den{n}"] == 0.0):
            return False
        if not np.all(np.isnan(r[f"xi{n}"])):
            return False
        if not np.all(np.isfinite(r[f"num{n}"])):
            return False
    return True


def check_slab_decomposition(o) -> bool:
    """Reading 14: a zero-outside box cut into 2 and 3 slabs along z, each
    slab a box of its own (origin shifted) holding its owned planes plus a
    halo of max|m_z| planes on either side (clipped at the faces), summed
    over its owned planes with the whole catalog's alpha: the slabs' num and
    den add up to the undivided box's (Eq. 19), which the brute-force pins
    fix."""
    g = GridSpec((10, 9, 18), (0.0, 0.0, 0.0), 1.0, False)
    rng = _rng(41)
    cd = np.stack([rng.integers(2, 8, 70), rng.integers(2, 7, 70), rng.integers(2, 16, 70)], 1)
    cr = np.stack([rng.integers(2, 8, 500), rng.integers(2, 7, 500), rng.integers(2, 16, 500)], 1)
    data, rand = lattice_catalog(g, cd), lattice_catalog(g, cr)
    shells = (1.5, 2.5)
    whole = o.correlate(g, shells, 1.0, data, rand, orders=(2, 3), engine="direct")
    halo = int(max(np.abs(o.shell_offsets(s, 1.0, 1.0))[:, 2].max() for s in shells))
    for parts in (2, 3):
        edges = np.linspace(0, 18, parts + 1).astype(int)
        num = {n: 0.0 for n in (2, 3)}
        den = {n: 0.0 for n in (2, 3)}
        for z0, z1 in zip(edges[:-1], edges[1:]):
            lo, hi = max(0, z0 - halo), min(18, z1 + halo)
            gs = GridSpec((10, 9, hi - lo), (0.0, 0.0, float(lo)), 1.0, False)
            r = o.correlate(gs, shells, 1.0, data, rand, orders=(2, 3), engine="direct",
                            alpha=whole["alpha"], owned_z=(z0 - lo, z1 - lo))
            for n in (2, 3):
                num[n] = num[n] + r[f"num{n}"]
                den[n] = den[n] + r[f"den{n}"]
        for n in (2, 3):
            if not (np.allclose(num[n], whole[f"num{n}"], rtol=1e-12, atol=1e-9)
                    and np.allclose(den[n], whole[f"den{n}"], rtol=1e-12, atol=1e-9)):
                return False
    return True


ALL_CHECKS = [
    check_lattice_gridding, check_out_of_grid, check_alpha_and_fields, check_shell_counts,
    check_intersect_rule, check_kernel_spectrum, check_pair_counts, check_triplet_counts,
    check_product_sums_high_order, check_signed_pairs, check_delta_response, check_fft_engine,
    check_constant_field_den, check_relabel_shells, check_translation, check_linearity,
    check_region_additivity, check_diagonal, check_sum_of_w, check_sampled_cells,
    check_multisets, check_guard_band, check_pair_sums_fft, check_grid_weights, check_sky_coordinates,
    check_factorised_randoms, check_delta_field, check_field_sums, check_product_map,
    check_periodic_support, check_xi_nonpositive_den, check_slab_decomposition,
]
