"""Loads (building on first use) the oracle's plain-C helpers.

TEST INFRASTRUCTURE ONLY.  The shared object is compiled with the host gcc
from oracle/fdint.c into oracle/_build/; it is independent of the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdint.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_fd.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/fdint.c into a shared object (gcc -O2 -fopenmp)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            L.oracle_fd_integrals.argtypes = [dp, ctypes.c_long, dp, dp, dp]
            L.oracle_fd_integrals.restype = None
            L.oracle_fd_inverse_half.argtypes = [dp, ctypes.c_long, dp, dp, ctypes.c_double]
            L.oracle_fd_inverse_half.restype = ctypes.c_long
            _lib = L
    return _lib
