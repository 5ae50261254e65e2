"""Thin ctypes binding of libconker.so (include/conker.h).

Argument marshalling only: every step of the correlation path runs in the
library's CUDA kernels.  Torch supplies device memory and streams: inputs may
be torch CUDA tensors (their data_ptr is passed), host numpy arrays (the
library stages them), and outputs are torch tensors allocated here.  If the
shared library is missing or does not load, every call raises: there is no
fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libconker.so")

CK_MAX_SHELLS = 64
CK_MAX_ORDER = 5

STATUS = {
    0: "CK_OK", 1: "CK_ERR_ARG", 2: "CK_ERR_BAD_POINTER", 3: "CK_ERR_OOM", 4: "CK_ERR_EMPTY_SHELL",
    5: "CK_ERR_KERNEL_TOO_LARGE", 6: "CK_ERR_GUARD_BAND", 7: "CK_ERR_ZERO_DENOM", 8: "CK_ERR_TIMEOUT",
    9: "CK_ERR_CUDA", 10: "CK_ERR_UNSUPPORTED", 11: "CK_ERR_NO_RANDOMS", 12: "CK_ERR_EMPTY_CATALOG",
}
RULES = {"center_bin": 0, "intersect": 1}
PRECISIONS = {"fp32": 0, "split_bf16": 1, "split_fp16": 2, "fp64": 3, "split_tf32": 4}


class CkError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        name = STATUS.get(self.code, str(code))
        msg = _lib().ck_status_string(self.code).decode() if _LIB is not None else name
        super().__init__(f"{where}: {name} ({msg})")


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("origin", ctypes.c_double * 3), ("cell", ctypes.c_double),
                ("periodic", ctypes.c_int32)]


class _Cosmology(ctypes.Structure):
    _fields_ = [("h0", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_k", ctypes.c_double),
                ("omega_l", ctypes.c_double), ("c", ctypes.c_double), ("z_max", ctypes.c_double)]


class _Selection(ctypes.Structure):
    _fields_ = [("n_tot", ctypes.c_double), ("p_ang", ctypes.POINTER(ctypes.c_double)), ("n_ra", ctypes.c_int32),
                ("n_dec", ctypes.c_int32), ("p_z", ctypes.POINTER(ctypes.c_double)), ("n_z", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("z_lo", ctypes.c_double), ("z_hi", ctypes.c_double)]


class _Shells(ctypes.Structure):
    _fields_ = [("n_shells", ctypes.c_int32), ("radius", ctypes.POINTER(ctypes.c_double)),
                ("width", ctypes.c_double), ("rule", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("spec_pitch", ctypes.c_int32), ("n_shells", ctypes.c_int32),
                ("max_order", ctypes.c_int32), ("max_offset", ctypes.c_int32 * 3),
                ("shell_size", ctypes.c_int64 * CK_MAX_SHELLS), ("n_multisets", ctypes.c_int64 * (CK_MAX_ORDER + 1)),
                ("workspace_bytes", ctypes.c_size_t), ("bank_stride", ctypes.c_int64),
                ("fused", ctypes.c_int32), ("fft_n", ctypes.c_int32 * 3)]


CK_STAGES = 15


class _StageTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * CK_STAGES), ("launches", ctypes.c_int64 * CK_STAGES),
                ("bytes", ctypes.c_double * CK_STAGES)]


class _Outputs(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_void_p * (CK_MAX_ORDER + 1)), ("num", ctypes.c_void_p * (CK_MAX_ORDER + 1)),
                ("den", ctypes.c_void_p * (CK_MAX_ORDER + 1)), ("dropped", ctypes.c_void_p)]


class _Catalog(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("plan", ctypes.c_int32)]


_LIB = None

# (name, restype, argtypes) for every entry point declared in include/conker.h
_P = ctypes.c_void_p
_SIGS = [
    ("ck_abi_version", ctypes.c_int32, []),
    ("ck_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ck_plan_workspace_size", ctypes.c_int, [ctypes.POINTER(_Grid), ctypes.POINTER(_Shells), ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    ("ck_plan_create", ctypes.c_int, [ctypes.POINTER(_Grid), ctypes.POINTER(_Shells), ctypes.c_int32, ctypes.c_int32,
                                      _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("ck_plan_destroy", ctypes.c_int, [_P]),
    ("ck_plan_get_info", ctypes.c_int, [_P, ctypes.POINTER(_Info)]),
    ("ck_set_randoms", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    ("ck_compute", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_Outputs), _P]),
    ("ck_set_randoms_diagonal", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    ("ck_sky_to_cartesian", ctypes.c_int, [ctypes.POINTER(_Cosmology), _P, _P, _P, ctypes.c_int64, _P, _P, _P,
                                           _P]),
    ("ck_set_randoms_weighted", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    ("ck_set_randoms_factorised", ctypes.c_int, [_P, ctypes.POINTER(_Cosmology), ctypes.POINTER(_Selection), _P]),
    ("ck_compute_weighted", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.POINTER(_Outputs), _P]),
    ("ck_compute_diagonal", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_Outputs),
                                           _P]),
    ("ck_compute_continuous", ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(_Outputs), _P]),
    ("ck_compute_cross", ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(_Outputs), _P]),
    ("ck_product_map", ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    ("ck_batch_compute", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(_Catalog), ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(_Outputs), _P]),
    ("ck_plan_status", ctypes.c_int, [_P, _P]),
    ("ck_plan_set_region", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]),
    ("ck_plan_autotune", ctypes.c_int, [_P, _P]),
    ("ck_plan_get_tuning", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    ("ck_plan_set_tuning", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    ("ck_get_grids", ctypes.c_int, [_P, _P, _P, _P]),
    ("ck_get_field", ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    ("ck_get_bank", ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    ("ck_get_kernel_spectrum", ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    ("ck_fft_r2c", ctypes.c_int, [_P, _P, _P, _P]),
    ("ck_fft_c2r", ctypes.c_int, [_P, _P, _P, _P]),
    ("ck_contract", ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_P), _P]),
    ("ck_contract_static", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(_P), _P]),
    ("ck_debug_force_timeout", ctypes.c_int, [ctypes.c_int64]),
    ("ck_profile_enable", ctypes.c_int, [_P, ctypes.c_int32]),
    ("ck_profile_read", ctypes.c_int, [_P, ctypes.POINTER(_StageTimes)]),
    ("ck_stage_name", ctypes.c_char_p, [ctypes.c_int32]),
]


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def load():
    """Load the library (raises if it is missing)."""
    return _lib()


def exported_symbols() -> Sequence[str]:
    return [s[0] for s in _SIGS]


def _check(code: int, where: str):
    if code != 0:
        raise CkError(code, where)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a):
    """data pointer of a torch tensor or a numpy array (host)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())


def _as_f32(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    torch = _torch()
    assert a.dtype == torch.float32 and a.is_contiguous(), "positions must be contiguous float32"
    return a


def sky_to_cartesian(ra_deg, dec_deg, redshift, h0: float = 100.0, omega_m: float = 0.307,
                     omega_k: float = 0.0, omega_l: float = 0.693, c: float = 300000.0, z_max: Optional[float] = None,
                     stream=None):
    """Sky coordinates (degrees, redshift; device float32 tensors) to the
    Cartesian frame of Eqs. 3-6 (ck_sky_to_cartesian): returns device float32
    tensors X, Y, Z.  z_max (default: the largest redshift) sets the distance
    table's range; points outside [0, z_max] get NaN.  The defaults are the
    paper's fiducial cosmology (Sec. 3), distances in h^-1 Mpc."""
    torch = _torch()
    ra, dec, z = _as_f32(ra_deg), _as_f32(dec_deg), _as_f32(redshift)
    n = int(z.shape[0])
    if z_max is None:
        z_max = float(z.max().item()) if n else 1.0
    cosmo = _Cosmology(float(h0), float(omega_m), float(omega_k), float(omega_l), float(c), float(z_max))
    X, Y, Z = (torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3))
    _check(_lib().ck_sky_to_cartesian(ctypes.byref(cosmo), _ptr(ra), _ptr(dec), _ptr(z), n, _ptr(X), _ptr(Y),
                                      _ptr(Z), _stream_ptr(stream)), "ck_sky_to_cartesian")
    return X, Y, Z


def contract_static(w0, bank, bank_stride: int, n_cells: int, n_shells: int, orders=(2, 3), stream=None):
    """ck_contract_static: the summation without a plan or any device
    allocation by the library (outputs are torch tensors allocated here)."""
    torch = _torch()
    sums = {n: torch.empty(math.comb(n_shells + n - 2, n - 1), dtype=torch.float64, device="cuda") for n in orders}
    arr = (ctypes.c_void_p * (CK_MAX_ORDER + 1))()
    for n, t in sums.items():
        arr[n] = t.data_ptr()
    _check(_lib().ck_contract_static(_ptr(w0), _ptr(bank), int(bank_stride), int(n_cells), int(n_shells),
                                     order_mask(orders), arr, _stream_ptr(stream)), "ck_contract_static")
    return sums


def force_timeout(ns: int = 0):
    """ck_debug_force_timeout: make the register contraction's consumer waits
    run out after ns nanoseconds on an mbarrier nothing arrives at (ns > 0),
    or restore normal operation (ns <= 0), on the current device."""
    _check(_lib().ck_debug_force_timeout(int(ns)), "ck_debug_force_timeout")


def order_mask(orders: Iterable[int]) -> int:
    m = 0
    for n in orders:
        m |= 1 << int(n)
    return m


class Plan:
    """A ck_plan: one grid, one shell bank, orders up to max_order."""

    def __init__(self, n: Sequence[int], origin: Sequence[float], cell: float, periodic: bool,
                 radii: Sequence[float], width: float, max_order: int = 3, rule: str = "center_bin",
                 precision: str = "fp32", workspace: str = "torch", stream=None, padded: bool = False):
        """padded=True (a non-periodic box): transform on a zero-padded grid
        (CK_GRID_PADDED); grids, fields and banks then have that grid's shape."""
        torch = _torch()
        lib = _lib()
        self._grid = _Grid((ctypes.c_int32 * 3)(*[int(v) for v in n]), (ctypes.c_double * 3)(*[float(v) for v in origin]),
                           float(cell), 2 if padded else (1 if periodic else 0))
        self._radii = (ctypes.c_double * len(radii))(*[float(r) for r in radii])
        self._shells = _Shells(len(radii), self._radii, float(width), RULES[rule])
        self.max_order = int(max_order)
        self.n_shells = len(radii)
        prec = PRECISIONS[precision]
        self._ws = None
        ws_ptr, ws_bytes = None, 0
        if workspace == "torch":
            nbytes = ctypes.c_size_t(0)
            _check(lib.ck_plan_workspace_size(ctypes.byref(self._grid), ctypes.byref(self._shells), self.max_order,
                                              prec, ctypes.byref(nbytes)), "ck_plan_workspace_size")
            self._ws = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            ws_ptr = ctypes.c_void_p((base + 255) // 256 * 256)
            ws_bytes = int(nbytes.value)
        h = ctypes.c_void_p()
        _check(lib.ck_plan_create(ctypes.byref(self._grid), ctypes.byref(self._shells), self.max_order, prec, ws_ptr,
                                  ws_bytes, _stream_ptr(stream), ctypes.byref(h)), "ck_plan_create")
        self._h = h
        info = _Info()
        _check(lib.ck_plan_get_info(self._h, ctypes.byref(info)), "ck_plan_get_info")
        self.n_cells = int(info.n_cells)
        self.spec_pitch = int(info.spec_pitch)
        self.max_offset = tuple(int(v) for v in info.max_offset)
        self.shell_size = [int(info.shell_size[s]) for s in range(self.n_shells)]
        self.n_multisets = {k: int(info.n_multisets[k]) for k in range(2, self.max_order + 1)}
        self.workspace_bytes = int(info.workspace_bytes)
        self.bank_stride = int(info.bank_stride)
        self.fused = bool(info.fused)
        self.fft_n = tuple(int(v) for v in info.fft_n)
        self.shape = (self.fft_n[2], self.fft_n[1], self.fft_n[0])
        self.box_shape = (int(n[2]), int(n[1]), int(n[0]))  # the caller's box, (nz, ny, nx)

    def close(self):
        if getattr(self, "_h", None):
            _lib().ck_plan_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the path ----------------------------------------------------------
    def set_randoms(self, x, y, z, stream=None, w=None):
        """Grid the randoms (ck_set_randoms; with weights w: ck_set_randoms_weighted)."""
        x, y, z = _as_f32(x), _as_f32(y), _as_f32(z)
        if w is None:
            _check(_lib().ck_set_randoms(self._h, _ptr(x), _ptr(y), _ptr(z), int(x.shape[0]), _stream_ptr(stream)),
                   "ck_set_randoms")
        else:
            w = _as_f32(w)
            _check(_lib().ck_set_randoms_weighted(self._h, _ptr(x), _ptr(y), _ptr(z), _ptr(w), int(x.shape[0]),
                                                  _stream_ptr(stream)), "ck_set_randoms_weighted")

    def set_randoms_factorised(self, n_tot: float, p_ang, p_z, z_lo: float, z_hi: float, h0: float = 100.0,
                               omega_m: float = 0.307, omega_k: float = 0.0, omega_l: float = 0.693,
                               c: float = 300000.0, z_max: Optional[float] = None, stream=None):
        """ck_set_randoms_factorised: the randoms field of Eq. 7 from the
        angular density p_ang (per steradian; shape (n_dec, n_ra), declination
        rows from -90, right-ascension columns from 0) and the redshift density
        p_z (per unit z, n_z bins of [z_lo, z_hi)); z_max (default z_hi) is the
        distance table's range.  Defaults: the paper's fiducial cosmology."""
        import numpy as np
        pa = np.ascontiguousarray(np.asarray(p_ang, np.float64))
        pz = np.ascontiguousarray(np.asarray(p_z, np.float64).ravel())
        if pa.ndim != 2:
            raise ValueError("p_ang must be 2-D (n_dec, n_ra)")
        cosmo = _Cosmology(float(h0), float(omega_m), float(omega_k), float(omega_l), float(c),
                           float(z_hi if z_max is None else z_max))
        dptr = ctypes.POINTER(ctypes.c_double)
        sel = _Selection(float(n_tot), pa.ctypes.data_as(dptr), int(pa.shape[1]), int(pa.shape[0]),
                         pz.ctypes.data_as(dptr), int(pz.shape[0]), 0, float(z_lo), float(z_hi))
        _check(_lib().ck_set_randoms_factorised(self._h, ctypes.byref(cosmo), ctypes.byref(sel),
                                                _stream_ptr(stream)), "ck_set_randoms_factorised")

    def set_randoms_diagonal(self, x, y, z, stream=None):
        """ck_set_randoms_diagonal: only the (s, .., s) denominators (for compute_diagonal)."""
        x, y, z = _as_f32(x), _as_f32(y), _as_f32(z)
        _check(_lib().ck_set_randoms_diagonal(self._h, _ptr(x), _ptr(y), _ptr(z), int(x.shape[0]),
                                              _stream_ptr(stream)), "ck_set_randoms_diagonal")

    def compute(self, x, y, z, orders=(2, 3), out: str = "device", stream=None, want=("xi", "num", "den"),
                outputs: Optional[Dict[str, Dict[int, object]]] = None, w=None) -> Dict[str, object]:
        """One catalog; returns {'xi': {n: T}, 'num': ..., 'den': ..., 'dropped': T} with dense
        [N_s]^(n-1) float64 tensors on the device (out='device') or in host memory (out='host')."""
        torch = _torch()
        x, y, z = _as_f32(x), _as_f32(y), _as_f32(z)
        ns = self.n_shells
        res: Dict[str, object] = {k: {} for k in ("xi", "num", "den")}
        o = _Outputs()
        dev = "cuda" if out == "device" else "cpu"
        for n in orders:
            if not 2 <= int(n) <= CK_MAX_ORDER:
                continue  # the library rejects the order mask
            for key in want:
                if outputs is not None:
                    t = outputs[key][n]
                else:
                    t = torch.empty((ns,) * (n - 1), dtype=torch.float64, device=dev, pin_memory=(dev == "cpu"))
                res[key][n] = t
                getattr(o, key)[n] = t.data_ptr()
        if outputs is not None and "dropped" in outputs:
            dropped = outputs["dropped"]
        else:
            dropped = torch.zeros(2, dtype=torch.int64, device=dev)
        o.dropped = dropped.data_ptr()
        res["dropped"] = dropped
        if w is None:
            code = _lib().ck_compute(self._h, _ptr(x), _ptr(y), _ptr(z), int(x.shape[0]), order_mask(orders),
                                     ctypes.byref(o), _stream_ptr(stream))
        else:  # weighted histogram of the data (ck_compute_weighted)
            w = _as_f32(w)
            code = _lib().ck_compute_weighted(self._h, _ptr(x), _ptr(y), _ptr(z), _ptr(w), int(x.shape[0]),
                                              order_mask(orders), ctypes.byref(o), _stream_ptr(stream))
        res["status"] = int(code)
        if code not in (0, 7):  # a zero denominator still fills the outputs (NaN there)
            raise CkError(code, "ck_compute")
        return res

    def _field_outputs(self, orders, out):
        torch = _torch()
        dev = "cuda" if out == "device" else "cpu"
        res: Dict[str, object] = {k: {} for k in ("xi", "num", "den")}
        o = _Outputs()
        for n in orders:
            for key in ("xi", "num", "den"):
                t = torch.empty((self.n_shells,) * (int(n) - 1), dtype=torch.float64, device=dev,
                                pin_memory=(dev == "cpu"))
                res[key][n] = t
                getattr(o, key)[n] = t.data_ptr()
        return res, o

    def _box_field(self, f):
        f = _as_f32(f)
        assert tuple(f.shape) == self.box_shape or int(np.prod(f.shape)) == int(np.prod(self.box_shape)), \
            "fields have the box's shape (nz, ny, nx)"
        return f

    def compute_continuous(self, d, r=None, orders=(2, 3), out: str = "device", stream=None) -> Dict[str, object]:
        """ck_compute_continuous (Eqs. 15-17): delta = (d - r) / r (r None: d
        is delta), xi_n = sum W_0 W_s1 .. with no denominator.  d, r: box-shaped
        float32 (device tensors or host arrays)."""
        d = self._box_field(d)
        r = None if r is None else self._box_field(r)
        res, o = self._field_outputs(orders, out)
        code = _lib().ck_compute_continuous(self._h, _ptr(d), _ptr(r), order_mask(orders), ctypes.byref(o),
                                            _stream_ptr(stream))
        res["status"] = int(code)
        _check(code, "ck_compute_continuous")
        return res

    def compute_cross(self, f0, f1, orders=(2, 3), out: str = "device", stream=None) -> Dict[str, object]:
        """ck_compute_cross (Sec. 2.8): W_0 = f0, W_s = f1 *** K_s."""
        f0, f1 = self._box_field(f0), self._box_field(f1)
        res, o = self._field_outputs(orders, out)
        code = _lib().ck_compute_cross(self._h, _ptr(f0), _ptr(f1), order_mask(orders), ctypes.byref(o),
                                       _stream_ptr(stream))
        res["status"] = int(code)
        _check(code, "ck_compute_cross")
        return res

    def product_map(self, shell: int, out: str = "device", stream=None):
        """ck_product_map: W_0 W_s / <B_0 B_s> per cell of the box for the last
        catalog (box-shaped float32, on the device or in host memory)."""
        if out == "device":
            torch = _torch()
            m = torch.empty(self.box_shape, dtype=torch.float32, device="cuda")
        else:
            m = np.empty(self.box_shape, dtype=np.float32)
        _check(_lib().ck_product_map(self._h, int(shell), _ptr(m), _stream_ptr(stream)), "ck_product_map")
        return m

    def compute_diagonal(self, x, y, z, orders=(2, 3), out: str = "device", stream=None) -> Dict[str, object]:
        """The equidistant functions of Eq. 14 only (ck_compute_diagonal): returns
        {'xi': {n: T}, 'num': ..., 'den': ..., 'dropped': T} with [N_s] float64 tensors,
        entry s = the multiset (s, .., s)."""
        torch = _torch()
        x, y, z = _as_f32(x), _as_f32(y), _as_f32(z)
        ns = self.n_shells
        res: Dict[str, object] = {k: {} for k in ("xi", "num", "den")}
        o = _Outputs()
        dev = "cuda" if out == "device" else "cpu"
        for n in orders:
            if not 2 <= int(n) <= CK_MAX_ORDER:
                continue  # the library rejects the order mask
            for key in ("xi", "num", "den"):
                t = torch.empty(ns, dtype=torch.float64, device=dev, pin_memory=(dev == "cpu"))
                res[key][n] = t
                getattr(o, key)[n] = t.data_ptr()
        dropped = torch.zeros(2, dtype=torch.int64, device=dev)
        o.dropped = dropped.data_ptr()
        res["dropped"] = dropped
        code = _lib().ck_compute_diagonal(self._h, _ptr(x), _ptr(y), _ptr(z), int(x.shape[0]), order_mask(orders),
                                          ctypes.byref(o), _stream_ptr(stream))
        res["status"] = int(code)
        if code not in (0, 7):  # a zero denominator still fills the outputs (NaN there)
            raise CkError(code, "ck_compute_diagonal")
        return res

    def set_region(self, z_begin: int, z_end: int, alpha: float = 0.0):
        """ck_plan_set_region: sums over box planes z_begin <= z < z_end,
        with the whole catalog's alpha (> 0) for a region of a decomposition."""
        _check(_lib().ck_plan_set_region(self._h, int(z_begin), int(z_end), float(alpha)), "ck_plan_set_region")

    def autotune(self, stream=None) -> Dict[str, int]:
        """ck_plan_autotune (after set_randoms or a compute): time the launch-shape choices
        on this plan's buffers and keep the fastest; returns them."""
        _check(_lib().ck_plan_autotune(self._h, _stream_ptr(stream)), "ck_plan_autotune")
        return self.tuning()

    def set_tuning(self, fwd_cols: int = 8, zreg_cols: int = 8, yinv_cols: int = 8, tc_ctas_per_sm: int = 2,
                   tc_stack_cols: int = 32, tc_thin_overlap: int = 1, z_direct: int = 1):
        arr = (ctypes.c_int32 * 7)(fwd_cols, zreg_cols, yinv_cols, tc_ctas_per_sm, tc_stack_cols, tc_thin_overlap,
                                   z_direct)
        _check(_lib().ck_plan_set_tuning(self._h, arr), "ck_plan_set_tuning")

    def tuning(self) -> Dict[str, int]:
        out = (ctypes.c_int32 * 8)()
        _check(_lib().ck_plan_get_tuning(self._h, out), "ck_plan_get_tuning")
        return dict(fwd_cols=out[0], zreg_cols=out[1], yinv_cols=out[2], tc_ctas_per_sm=out[3],
                    tc_stack_cols=out[4], tc_thin_overlap=out[5], z_direct=out[6], tuned=bool(out[7]))

    def status(self, stream=None) -> int:
        return int(_lib().ck_plan_status(self._h, _stream_ptr(stream)))

    # -- per-stage event timing -------------------------------------------
    def profile(self, enable: bool = True):
        _check(_lib().ck_profile_enable(self._h, 1 if enable else 0), "ck_profile_enable")

    def profile_read(self) -> Dict[str, Dict[str, float]]:
        t = _StageTimes()
        _check(_lib().ck_profile_read(self._h, ctypes.byref(t)), "ck_profile_read")
        out = {}
        for i in range(CK_STAGES):
            if t.launches[i]:
                out[_lib().ck_stage_name(i).decode()] = dict(ms=float(t.ms[i]), launches=int(t.launches[i]),
                                                             bytes=float(t.bytes[i]))
        return out

    # -- stage access ------------------------------------------------------
    def grids(self, stream=None):
        torch = _torch()
        d = torch.empty(self.shape, dtype=torch.int32, device="cuda")
        r = torch.empty(self.shape, dtype=torch.int32, device="cuda")
        _check(_lib().ck_get_grids(self._h, _ptr(d), _ptr(r), _stream_ptr(stream)), "ck_get_grids")
        return d, r

    def field(self, which: int, stream=None):
        torch = _torch()
        f = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check(_lib().ck_get_field(self._h, int(which), _ptr(f), _stream_ptr(stream)), "ck_get_field")
        return f

    def bank(self, shell: int, stream=None):
        torch = _torch()
        f = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check(_lib().ck_get_bank(self._h, int(shell), _ptr(f), _stream_ptr(stream)), "ck_get_bank")
        return f

    def kernel_spectrum(self, shell: int, stream=None):
        torch = _torch()
        nz, ny, nx = self.shape
        f = torch.empty((nz // 2 + 1, ny // 2 + 1, nx // 2 + 1), dtype=torch.float32, device="cuda")
        _check(_lib().ck_get_kernel_spectrum(self._h, int(shell), _ptr(f), _stream_ptr(stream)),
               "ck_get_kernel_spectrum")
        return f

    def fft_r2c(self, real, stream=None):
        torch = _torch()
        nz, ny, nx = self.shape
        spec = torch.empty((nz, ny, self.spec_pitch), dtype=torch.complex64, device="cuda")
        _check(_lib().ck_fft_r2c(self._h, _ptr(real), _ptr(spec), _stream_ptr(stream)), "ck_fft_r2c")
        return spec

    def fft_c2r(self, spec, stream=None):
        torch = _torch()
        out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        _check(_lib().ck_fft_c2r(self._h, _ptr(spec), _ptr(out), _stream_ptr(stream)), "ck_fft_c2r")
        return out

    def contract(self, w0, bank, bank_stride: int, orders=(2, 3), stream=None):
        torch = _torch()
        sums = {n: torch.empty(self.n_multisets[n], dtype=torch.float64, device="cuda") for n in orders}
        arr = (ctypes.c_void_p * (CK_MAX_ORDER + 1))()
        for n, t in sums.items():
            arr[n] = t.data_ptr()
        _check(_lib().ck_contract(self._h, _ptr(w0), _ptr(bank), int(bank_stride), order_mask(orders), arr,
                                  _stream_ptr(stream)), "ck_contract")
        return sums


def batch_compute(plans, catalogs, orders=(2, 3), out: str = "device", stream=None,
                  want=("xi", "num", "den")):
    """ck_batch_compute: catalogs is a sequence of (x, y, z, plan_index) with
    device float32 positions; returns one result dict per catalog, as
    Plan.compute does (dense [N_s]^(n-1) float64 tensors)."""
    torch = _torch()
    lib = _lib()
    hs = (_P * len(plans))(*[p._h for p in plans])
    cats = (_Catalog * max(1, len(catalogs)))()
    outs = (_Outputs * max(1, len(catalogs)))()
    dev = "cuda" if out == "device" else "cpu"
    keep, results = [], []
    for i, (x, y, z, j) in enumerate(catalogs):
        x, y, z = _as_f32(x), _as_f32(y), _as_f32(z)
        keep.append((x, y, z))
        cats[i].x, cats[i].y, cats[i].z = _ptr(x), _ptr(y), _ptr(z)
        cats[i].n = int(x.shape[0])
        cats[i].plan = int(j)
        ns = plans[j].n_shells if 0 <= int(j) < len(plans) else plans[0].n_shells  # the library rejects a bad index
        res = {k: {} for k in ("xi", "num", "den")}
        for n in orders:
            if not 2 <= int(n) <= CK_MAX_ORDER:
                continue
            for key in want:
                t = torch.empty((ns,) * (n - 1), dtype=torch.float64, device=dev, pin_memory=(dev == "cpu"))
                res[key][n] = t
                getattr(outs[i], key)[n] = t.data_ptr()
        d = torch.zeros(2, dtype=torch.int64, device=dev)
        outs[i].dropped = d.data_ptr()
        res["dropped"] = d
        results.append(res)
    code = lib.ck_batch_compute(hs, len(plans), cats, len(catalogs), order_mask(orders), outs, _stream_ptr(stream))
    if code not in (0, 7):
        raise CkError(code, "ck_batch_compute")
    for r in results:
        r["status"] = int(code)
    return results
