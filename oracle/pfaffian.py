"""ctypes front end of oracle/pfaffian.c (plain Parlett-Reid Pfaffian).

Pinned (tests/test_oracle_pfaffian.py): explicit 2x2 and 4x4 formulas,
Pf^2 = det (numpy.linalg.det), Pf(B A B^T) = det(B) Pf(A), block-diagonal
products, Pf(J) = 1, and a brute-force sum over perfect matchings for 6x6.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfaffian.c")
_LIB = os.path.join(_HERE, "_oracle_pfaffian.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C Pfaffian with gcc (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_pfaffian_z.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p]
        lib.oracle_pfaffian_d.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        _lib = lib
    return _lib


def log_pfaffian(A: np.ndarray):
    """Return (log|Pf A|, phase) with phase a unit complex (real +-1 for real A)."""
    lib = _load()
    n = A.shape[0]
    la = ctypes.c_double()
    if np.iscomplexobj(A):
        buf = np.ascontiguousarray(A, dtype=np.complex128).copy()
        ph = np.zeros(1, dtype=np.complex128)
        lib.oracle_pfaffian_z(n, buf.ctypes.data, ctypes.byref(la), ph.ctypes.data)
        return la.value, complex(ph[0])
    buf = np.ascontiguousarray(A, dtype=np.float64).copy()
    sg = ctypes.c_double()
    lib.oracle_pfaffian_d(n, buf.ctypes.data, ctypes.byref(la), ctypes.byref(sg))
    return la.value, float(sg.value)


def pfaffian(A: np.ndarray):
    la, ph = log_pfaffian(A)
    return ph * np.exp(la)
