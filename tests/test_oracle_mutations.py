"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins catch each one: a dropped term, a wrong sign, an off-by-one, transposed
axes, a wrong boundary rule."""
import numpy as np
import pytest

import oracle.conker_oracle as O
from tests import oracle_pins as P


def _any_fails(monkeypatch, name, fn, checks=None):
    monkeypatch.setattr(O, name, fn)
    checks = checks or P.ALL_CHECKS
    for c in checks:
        try:
            if not c(O):
                return True
        except Exception:
            return True
    return False


_orig_density = O.density_fields
_orig_index = O.cell_index
_orig_counts = O.grid_counts
_orig_shell = O.shell_offsets
_orig_psums = O.product_sums
_orig_conv = O.convolve_direct
_orig_fft = O.convolve_fft


def wrong_sign_density(D, R):
    a, N, Rt = _orig_density(D, R)
    return a, D.astype(np.float64) + a * R.astype(np.float64), Rt


def off_by_one_index(x, origin, cell):
    return _orig_index(x, origin, cell) + 1


def transposed_counts(x, y, z, grid):
    return _orig_counts(y, x, z, grid)


def closed_shell(radius, width, cell, rule="center_bin"):
    # includes the outer bound (<= instead of <)
    if rule != "center_bin":
        return _orig_shell(radius, width, cell, rule)
    return _orig_shell(radius, width + 1e-9, cell, rule)


def dropped_w0(W0, W, order):
    return _orig_psums(np.ones_like(W0), W, order)


def dropped_offset(F, offsets, periodic):
    return _orig_conv(F, offsets[1:], periodic)


def fft_no_conj_shift(F, offsets):
    # off-by-one shift of the kernel grid
    return np.roll(_orig_fft(F, offsets), 1, axis=0)


_orig_quant = O.quantize_weights


def truncated_weights(w):
    # rounds toward zero instead of to nearest (ties to even)
    return np.trunc(np.asarray(w, np.float32).astype(np.float64) * 2.0 ** O.WEIGHT_FRAC_BITS).astype(np.int64)


def float32_weight_sums(x, y, z, w, grid):
    # sums the weights in float32 (order-dependent rounding)
    nx, ny, nz = (int(v) for v in grid.n)
    D, tot, dropped = _orig_gw(x, y, z, np.ones_like(np.asarray(w, np.float32)), grid)
    acc = np.zeros(nx * ny * nz, np.float32)
    k = [O.cell_index(c, o, grid.cell) for c, o in zip((x, y, z), grid.origin)]
    keep = np.isfinite(np.asarray(w, np.float32))
    for a, n in enumerate((nx, ny, nz)):
        keep &= (k[a] >= 0) & (k[a] < n)
    flat = (k[2][keep] * ny + k[1][keep]) * nx + k[0][keep]
    np.add.at(acc, flat, np.asarray(w, np.float32)[keep])
    return acc.astype(np.float64).reshape(nz, ny, nx), float(acc.sum()), dropped


_orig_gw = O.grid_weights
_orig_cd = O.comoving_distance


def curvature_dropped(z, h0, omega_m, omega_k, omega_l, c):
    # leaves out the curvature term of Eq. 3
    return _orig_cd(z, h0, omega_m, 0.0, omega_l, c)


def swapped_angles(ra_deg, dec_deg, z, h0, omega_m, omega_k, omega_l, c):
    # declination and right ascension exchanged in Eqs. 4-6
    r = _orig_cd(z, h0, omega_m, omega_k, omega_l, c)
    a = np.radians(np.asarray(dec_deg, np.float64))
    d = np.radians(np.asarray(ra_deg, np.float64))
    return r * np.cos(d) * np.cos(a), r * np.cos(d) * np.sin(a), r * np.sin(d)



_orig_fr = O.factorised_randoms_at


def flipped_declination(cells, grid, **sel):
    # declination bins counted from the north pole instead of the south
    return _orig_fr(cells, grid, **dict(sel, p_ang=np.asarray(sel["p_ang"])[::-1]))


def linear_jacobian(cells, grid, **sel):
    # dV_sph taken as r dr dOmega instead of r^2 dr dOmega
    ctr = np.asarray(grid.origin, np.float64) + (np.asarray(cells, np.float64).reshape(-1, 3) + 0.5) * grid.cell
    return _orig_fr(cells, grid, **sel) * np.sqrt((ctr * ctr).sum(axis=1))



_orig_fs = O.field_sums


def delta_over_data(D, R):
    # (D - R) / D instead of (D - R) / R
    D = np.asarray(D, np.float64)
    R = np.asarray(R, np.float64)
    out = np.zeros(D.shape)
    ok = (R > 0) & (D != 0)
    out[ok] = (D[ok] - R[ok]) / D[ok]
    return out


def cross_convolves_w0(grid, shells, width, W0, F, orders=(2, 3), engine="direct", rule="center_bin"):
    # W_s taken from W_0's field instead of the second tracer's
    return _orig_fs(grid, shells, width, W0, W0, orders, engine, rule)


def map_without_volume(W0, Ws, den2_s, n_box):
    # <B_0 B_s> taken as the sum instead of the average over the cells
    return np.asarray(W0, np.float64) * np.asarray(Ws, np.float64) / den2_s


_orig_support = O.check_periodic_support
_orig_xi = O.xi_from


def support_closed(offsets, n):
    # 2 max|m| <= n instead of < n
    if offsets.size == 0:
        return True
    m = np.abs(offsets).max(axis=0)
    return bool(all(2 * int(m[a]) <= int(n[a]) for a in range(3)))


def support_wrong_axis(offsets, n):
    # every axis tested against the x length
    return _orig_support(offsets, [n[0], n[0], n[0]])


def xi_keeps_negative(num, den):
    # NaN only where den == 0: a negative denominator gives a signed xi
    num = np.asarray(num, np.float64)
    den = np.asarray(den, np.float64)
    out = np.full(num.shape, np.nan)
    ok = den != 0
    out[ok] = num[ok] / den[ok]
    return out


def xi_divides_anyway(num, den):
    # no rule: num / den everywhere (inf or a signed value instead of NaN)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.asarray(num, np.float64) / np.asarray(den, np.float64)


_orig_corr = O.correlate


def slab_own_alpha(*a, **kw):
    # each region normalised by its own randoms instead of the whole catalog's
    kw.pop("alpha", None)
    return _orig_corr(*a, **kw)


def slab_halo_summed(*a, **kw):
    # the halo planes counted in the sums as well as the owned planes
    kw.pop("owned_z", None)
    return _orig_corr(*a, **kw)


MUTANTS = [
    ("density_fields", wrong_sign_density),
    ("cell_index", off_by_one_index),
    ("grid_counts", transposed_counts),
    ("shell_offsets", closed_shell),
    ("product_sums", dropped_w0),
    ("convolve_direct", dropped_offset),
    ("convolve_fft", fft_no_conj_shift),
    ("quantize_weights", truncated_weights),
    ("grid_weights", float32_weight_sums),
    ("comoving_distance", curvature_dropped),
    ("sky_to_cartesian", swapped_angles),
    ("factorised_randoms_at", flipped_declination),
    ("factorised_randoms_at", linear_jacobian),
    ("delta_field", delta_over_data),
    ("field_sums", cross_convolves_w0),
    ("product_map", map_without_volume),
    ("check_periodic_support", support_closed),
    ("check_periodic_support", support_wrong_axis),
    ("xi_from", xi_keeps_negative),
    ("xi_from", xi_divides_anyway),
    ("correlate", slab_own_alpha),
    ("correlate", slab_halo_summed),
]


@pytest.mark.parametrize("name,fn", MUTANTS, ids=[m[0] + ":" + m[1].__name__ for m in MUTANTS])
def test_mutant_is_caught(monkeypatch, name, fn):
    assert _any_fails(monkeypatch, name, fn)
