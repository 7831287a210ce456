"""ctypes loader for ``oracle/brute_force.c``.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  ``build()`` compiles
the C file into ``oracle/liboracle_brute.so`` with gcc; if the shared object
is missing it is compiled here on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brute_force.c")
_LIB = os.path.join(_HERE, "liboracle_brute.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the brute-force enumerator into a shared object (plain gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.oracle_brute_ln_z.restype = ctypes.c_double
        _lib.oracle_brute_ln_z.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]
    return _lib


def brute_ln_z(B: np.ndarray, w: np.ndarray, Lx: int, Ly: int) -> float:
    """ln Z by enumeration of all q^(Lx Ly) configurations."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = B.shape[0]
    lib = _load()
    r = lib.oracle_brute_ln_z(q, Lx, Ly,
                              B.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if not np.isfinite(r):
        raise ValueError("brute force rejected the input (too many states or non-positive weights)")
    return float(r)
