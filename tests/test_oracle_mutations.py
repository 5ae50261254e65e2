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


MUTANTS = [
    ("density_fields", wrong_sign_density),
    ("cell_index", off_by_one_index),
    ("grid_counts", transposed_counts),
    ("shell_offsets", closed_shell),
    ("product_sums", dropped_w0),
    ("convolve_direct", dropped_offset),
    ("convolve_fft", fft_no_conj_shift),
]


@pytest.mark.parametrize("name,fn", MUTANTS, ids=[m[0] + ":" + m[1].__name__ for m in MUTANTS])
def test_mutant_is_caught(monkeypatch, name, fn):
    assert _any_fails(monkeypatch, name, fn)
