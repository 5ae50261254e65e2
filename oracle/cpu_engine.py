"""Python access to the FP64 C++/OpenMP engine (conker_cpu.cpp).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: tests/ and bench.py's
CPU-baseline and reference legs use it.  ``build()`` compiles the engine in
place with g++ (-O3 -fopenmp); ``correlate`` runs the whole path for one
catalog and returns the same per-multiset sums as conker_oracle.correlate.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "conker_cpu.cpp")
LIB = os.path.join(HERE, "libconker_cpu.so")
_LIB = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp,
                        SRC], check=True, capture_output=True, text=True)
        os.replace(tmp, LIB)
    return LIB


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.cko_correlate.restype = ctypes.c_int
        lib.cko_correlate.argtypes = [P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, ctypes.c_double,
                                      ctypes.c_int, P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        lib.cko_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def threads() -> int:
    """OpenMP threads the engine uses (OMP_NUM_THREADS, else the cores)."""
    return int(_lib().cko_threads())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def correlate(grid, shells, width, data, randoms, orders=(2, 3), engine="fft", rule="center_bin", alpha=None,
              owned_z=None):
    """num{n}, den{n}, abs_num{n}, abs_den{n} (multiset order), alpha and
    the dropped counts, as conker_oracle.correlate returns them."""
    from math import comb
    n = np.array([int(v) for v in grid.n], np.int32)
    origin = np.array([float(v) for v in grid.origin], np.float64)
    rad = np.ascontiguousarray(np.asarray(shells, np.float64))
    ns = rad.size
    mask = 0
    for k in orders:
        mask |= 1 << int(k)
    total = sum(comb(ns + k - 2, k - 1) for k in range(2, 6) if (mask >> k) & 1)
    outs = [np.zeros(max(total, 1)) for _ in range(4)]
    a_out = np.zeros(1)
    dropped = np.zeros(2, np.int64)
    arrs = [np.ascontiguousarray(np.asarray(v, np.float32)) for v in (data.x, data.y, data.z, randoms.x, randoms.y,
                                                                       randoms.z)]
    z0, z1 = (int(owned_z[0]), int(owned_z[1])) if owned_z is not None else (0, 0)
    code = _lib().cko_correlate(_ptr(n), _ptr(origin), float(grid.cell), 1 if grid.periodic else 0, ns, _ptr(rad),
                                float(width), 0 if rule == "center_bin" else 1, _ptr(arrs[0]), _ptr(arrs[1]),
                                _ptr(arrs[2]), arrs[0].size, _ptr(arrs[3]), _ptr(arrs[4]), _ptr(arrs[5]), arrs[3].size,
                                mask, 0 if engine == "direct" else 1, float(alpha or 0.0), z0, z1,
                                *(_ptr(o) for o in outs), _ptr(a_out), _ptr(dropped))
    if code != 0:
        raise ValueError("cko_correlate rejected its arguments")
    res = dict(alpha=float(a_out[0]), dropped_d=int(dropped[0]), dropped_r=int(dropped[1]))
    base = 0
    for k in range(2, 6):
        if not (mask >> k) & 1:
            continue
        m = comb(ns + k - 2, k - 1)
        for key, o in zip(("num", "den", "abs_num", "abs_den"), outs):
            res[f"{key}{k}"] = o[base:base + m].copy()
        base += m
    return res
