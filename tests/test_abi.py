"""The C-ABI library without a GPU: it builds, loads, exports every entry
point declared in include/conker.h, and validates arguments on the host
(before any CUDA call) with the documented status codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "conker.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\**\s+\**(ck_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2108_00015_gb300 import conker
    return conker.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2108_00015_gb300 import conker
    assert sorted(conker.exported_symbols()) == names


def test_abi_version(lib):
    assert lib.ck_abi_version() == 1
    assert lib.ck_status_string(0) == b"ok"


def _ws(lib, n=(32, 32, 32), cell=10.0, periodic=1, radii=(20.0, 40.0), width=10.0, rule=0, max_order=3, prec=0):
    from paper_2108_00015_gb300.conker import _Grid, _Shells
    g = _Grid((ctypes.c_int32 * 3)(*n), (ctypes.c_double * 3)(0, 0, 0), cell, periodic)
    r = (ctypes.c_double * len(radii))(*radii)
    s = _Shells(len(radii), r, width, rule)
    b = ctypes.c_size_t(0)
    code = lib.ck_plan_workspace_size(ctypes.byref(g), ctypes.byref(s), max_order, prec, ctypes.byref(b))
    return code, b.value


def test_host_validation(lib):
    code, nbytes = _ws(lib)
    assert code == 0 and nbytes > 32 ** 3 * 4 * 8
    assert _ws(lib, n=(33, 32, 32))[0] == 10          # odd axis
    assert _ws(lib, n=(14, 32, 32))[0] == 10          # prime factor 7
    assert _ws(lib, n=(1024, 32, 32))[0] == 10        # beyond 512
    assert _ws(lib, cell=0.0)[0] == 1
    assert _ws(lib, max_order=6)[0] == 1
    assert _ws(lib, max_order=1)[0] == 1
    assert _ws(lib, prec=1)[0] == 0                   # split-BF16: bank + tensor-core blocked product
    assert _ws(lib, prec=2, max_order=5)[0] == 0      # split-FP16
    assert _ws(lib, prec=1)[1] > _ws(lib, prec=4)[1]  # the 16-bit forms keep the bank (no fused pass)
    assert _ws(lib, prec=4)[0] == 0                   # split-TF32, fused
    assert _ws(lib, prec=4, max_order=5)[0] == 0      # split-TF32, bank + tensor-core blocked product
    assert _ws(lib, prec=4, radii=tuple(20.0 + 5 * i for i in range(17)), width=5.0)[0] == 0
    assert _ws(lib, prec=5)[0] == 1
    assert _ws(lib, radii=(0.2,), width=0.1)[0] == 4  # no lattice offset in the shell
    assert _ws(lib, radii=(170.0,))[0] == 5           # reaches half of a 32-cell box
    assert _ws(lib, rule=7)[0] == 1
    assert _ws(lib, width=0.0)[0] == 1
    # zero-padded survey boxes (CK_GRID_PADDED): any box size whose padded length exists
    assert _ws(lib, n=(23, 17, 15), periodic=2, cell=8.0, radii=(16.0, 24.0), width=8.0)[0] == 0
    assert _ws(lib, n=(33, 32, 32), periodic=2)[0] == 0
    assert _ws(lib, n=(510, 32, 32), periodic=2)[0] == 10  # 510 + reach > 512
    padded = _ws(lib, n=(30, 30, 30), periodic=2)[1]
    assert padded > _ws(lib, n=(30, 30, 30), periodic=0)[1]  # transformed on a larger grid


def test_null_plan_entry_points(lib):
    """Entry points taking a plan reject a null one before any CUDA call."""
    from paper_2108_00015_gb300.conker import _Outputs
    o = _Outputs()
    for name in ("ck_compute", "ck_compute_diagonal"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_Outputs),
                                               ctypes.c_void_p]
        assert fn(None, None, None, None, 0, 4, ctypes.byref(o), None) == 2, name  # CK_ERR_BAD_POINTER
    for name in ("ck_compute_continuous", "ck_compute_cross"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32, ctypes.POINTER(_Outputs), ctypes.c_void_p]
        assert fn(None, None, None, 4, ctypes.byref(o), None) == 2, name
    fn = lib.ck_product_map
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    assert fn(None, 0, None, None) == 2
    fn = lib.ck_set_randoms_factorised
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 4
    assert fn(None, None, None, None) == 2


def test_sky_validation(lib):
    """ck_sky_to_cartesian checks its cosmology before any CUDA call."""
    from paper_2108_00015_gb300.conker import _Cosmology
    f = lib.ck_sky_to_cartesian
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(_Cosmology)] + [ctypes.c_void_p] * 3 + [ctypes.c_int64] + [ctypes.c_void_p] * 4
    ok = _Cosmology(100.0, 0.307, 0.0, 0.693, 300000.0, 1.0)
    assert f(ok, None, None, None, 0, None, None, None, None) == 0          # nothing to do
    assert f(None, None, None, None, 0, None, None, None, None) == 2        # CK_ERR_BAD_POINTER
    assert f(ok, None, None, None, -1, None, None, None, None) == 1         # CK_ERR_ARG
    assert f(ok, None, None, None, 5, None, None, None, None) == 2          # missing arrays
    for bad in (_Cosmology(0.0, 0.3, 0.0, 0.7, 3e5, 1.0), _Cosmology(100.0, 0.3, 0.0, 0.7, 3e5, -1.0),
                _Cosmology(100.0, 0.3, 0.0, -2.0, 3e5, 1.0), _Cosmology(100.0, float("nan"), 0.0, 0.7, 3e5, 1.0)):
        assert f(bad, None, None, None, 0, None, None, None, None) == 1



def test_factorised_validation(lib):
    """ck_set_randoms_factorised checks its cosmology and selection on the
    host before it touches the plan (a placeholder handle here)."""
    import numpy as np
    from paper_2108_00015_gb300.conker import _Cosmology, _Selection
    f = lib.ck_set_randoms_factorised
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Cosmology), ctypes.POINTER(_Selection), ctypes.c_void_p]
    handle = ctypes.create_string_buffer(64)
    dptr = ctypes.POINTER(ctypes.c_double)
    pa = np.full((3, 4), 0.1)
    pz = np.ones(5)

    def sel(n_tot=1e5, a=pa, z=pz, nra=4, ndec=3, nz=5, zlo=0.1, zhi=0.5):
        return _Selection(n_tot, a.ctypes.data_as(dptr), nra, ndec, z.ctypes.data_as(dptr), nz, 0, zlo, zhi)
    ok = _Cosmology(100.0, 0.307, 0.0, 0.693, 300000.0, 0.6)
    h = ctypes.cast(handle, ctypes.c_void_p)
    assert f(None, ok, sel(), None) == 2                                      # no plan
    assert f(h, None, sel(), None) == 2
    assert f(h, ok, None, None) == 2
    assert f(h, _Cosmology(100.0, 0.3, 0.0, -2.0, 3e5, 1.0), sel(), None) == 1
    assert f(h, ok, _Selection(1e5, None, 4, 3, pz.ctypes.data_as(dptr), 5, 0, 0.1, 0.5), None) == 2
    for bad in (sel(nra=0), sel(nz=0), sel(n_tot=float("nan")), sel(n_tot=-1.0), sel(zlo=-0.1),
                sel(zhi=0.1), sel(a=np.full((3, 4), -0.1)), sel(z=np.array([1.0, 1.0, np.inf, 1.0, 1.0])),
                sel(nra=1 << 14, ndec=1 << 13), sel(nz=(1 << 20) + 1)):
        assert f(h, ok, bad, None) == 1


def test_survey_workspace_fits(lib):
    # 512^3, 16 shells, orders <= 3.  Mixed (split-TF32, fused pass, no bank):
    # counts + field + spectrum + 16 scratch spectra + kernel octants + one field
    radii = tuple(30.0 + 8 * i for i in range(16))
    kw = dict(n=(512, 512, 512), cell=8.0, periodic=0, radii=radii, width=8.0, max_order=3)
    code, fused = _ws(lib, prec=4, **kw)
    assert code == 0
    assert 10e9 < fused < 15e9
    # plain FP32 keeps the 16-field bank (8.6 GB more)
    code, banked = _ws(lib, prec=0, **kw)
    assert code == 0
    assert abs((banked - fused) - 15 * 512 ** 3 * 4) < 0.05e9


def test_undersized_workspace(lib):
    """A caller workspace smaller than ck_plan_workspace_size reports is
    refused with CK_ERR_OOM before any CUDA call (the pointer is never
    touched, so a placeholder address serves)."""
    from paper_2108_00015_gb300.conker import _Grid, _Shells
    g = _Grid((ctypes.c_int32 * 3)(32, 32, 32), (ctypes.c_double * 3)(0, 0, 0), 10.0, 1)
    r = (ctypes.c_double * 2)(20.0, 40.0)
    s = _Shells(2, r, 10.0, 0)
    code, need = _ws(lib)
    assert code == 0
    out = ctypes.c_void_p(1)
    f = lib.ck_plan_create
    fake = ctypes.c_void_p(1 << 20)
    assert f(ctypes.byref(g), ctypes.byref(s), 3, 0, fake, need - 1, None, ctypes.byref(out)) == 3
    assert out.value is None
    assert f(ctypes.byref(g), ctypes.byref(s), 3, 0, fake, 0, None, ctypes.byref(out)) == 3


def test_tuning_entry_points_validate(lib):
    """ck_plan_autotune, ck_plan_set_tuning and ck_plan_get_tuning reject a
    null plan or array (CK_ERR_BAD_POINTER) before any CUDA call."""
    arr = (ctypes.c_int32 * 8)(8, 8, 16, 2, 32, 0, 0, 0)
    for name in ("ck_plan_autotune", "ck_plan_set_tuning", "ck_plan_get_tuning"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        assert fn(None, ctypes.cast(arr, ctypes.c_void_p)) == 2, name
    fn = lib.ck_plan_set_tuning
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: a null array is refused first
    assert fn(fake, None) == 2
    for bad in ((7, 8, 16, 2, 32, 0, 1), (8, 32, 16, 2, 32, 0, 1), (8, 8, 16, 0, 32, 0, 1), (8, 8, 16, 4, 32, 0, 1),
                (8, 8, 8, 2, -1, 0, 1), (8, 8, 8, 2, 129, 0, 1), (8, 8, 8, 2, 32, 2, 1), (8, 8, 8, 2, 32, 1, 2),
                (8, 8, 8, 2, 32, 1, -1)):
        # out-of-range choices are refused (CK_ERR_ARG) before the plan is read
        assert fn(fake, ctypes.cast((ctypes.c_int32 * 7)(*bad), ctypes.c_void_p)) == 1, bad
