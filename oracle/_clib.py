"""Build and load the oracle's C part (oracle/matern_ref.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "matern_ref.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile matern_ref.c with gcc (OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        _lib.oracle_besselk.restype = d
        _lib.oracle_besselk.argtypes = [d, d]
        _lib.oracle_besselk_scaled.restype = d
        _lib.oracle_besselk_scaled.argtypes = [d, d]
        _lib.oracle_matern.restype = d
        _lib.oracle_matern.argtypes = [d, d, d, d]
        _lib.oracle_matern_vec.restype = None
        _lib.oracle_matern_vec.argtypes = [i64, p, d, d, d, p]
        _lib.oracle_matern_matrix.restype = None
        _lib.oracle_matern_matrix.argtypes = [i64, p, d, d, d, p]
        _lib.oracle_matern_block.restype = None
        _lib.oracle_matern_block.argtypes = [i64, p, i64, p, d, d, d, p]
    return _lib


def ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)
