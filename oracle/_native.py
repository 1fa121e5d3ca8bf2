"""Builds and loads the oracle's plain-C part (``ora_core.c``).

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg load this library.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ora_core.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ora_core.c with gcc (OpenMP, no floating-point contraction)."""
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    out = os.path.join(_BUILD, f"libora_{tag}.so")
    if os.path.exists(out) and not force:
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.ora_apply_h.argtypes = [i64, i32, i32, P, P, f64, P, i32, P, P, P, P, f64, P, P]
            L.ora_apply_h.restype = i32
            L.ora_cholesky.argtypes = [i32, P, P]
            L.ora_cholesky.restype = i32
            L.ora_tri_inv_upper.argtypes = [i32, P, P]
            L.ora_tri_inv_upper.restype = i32
            L.ora_jacobi_eig.argtypes = [i32, P, P, P, i32, f64]
            L.ora_jacobi_eig.restype = i32
            _lib = L
    return _lib


def ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data
