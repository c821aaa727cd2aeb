"""Builds and loads the oracle's plain C direct-sum library (test infrastructure).

The shared object is compiled from ``oracle/direct.c`` with the host C
compiler into ``oracle/_build/`` on first use (or by ``build()``), and is
loaded with ctypes.  It has no relation to the CUDA library of the product.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_direct.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile direct.c (gcc, -O2, OpenMP) unless an up-to-date .so exists."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            L.oracle_interaction_tensor.argtypes = [ctypes.c_double] * 4 + [dp]
            L.oracle_interaction_tensor.restype = None
            L.oracle_direct_matvec.argtypes = [ctypes.c_int64, ip, dp, ctypes.c_double, dp, dp, ctypes.c_int]
            L.oracle_direct_matvec.restype = None
            L.oracle_direct_matvec_rows.argtypes = [ctypes.c_int64, ip, dp, ctypes.c_double, dp,
                                                    ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, dp,
                                                    ctypes.c_int]
            L.oracle_direct_matvec_rows.restype = None
            L.oracle_dense_matrix.argtypes = [ctypes.c_int64, ip, dp, ctypes.c_double, dp]
            L.oracle_dense_matrix.restype = None
            L.oracle_csca_double_sum.argtypes = [ctypes.c_int64, ip, ctypes.c_double, dp, ctypes.c_int]
            L.oracle_csca_double_sum.restype = ctypes.c_double
            _lib = L
        return _lib
