"""OpenMP FP32 lock-free CPU baseline of the training step (hogwild.c).

A timed comparison point for bench.py only (all host threads, FP32, Alg. 3
with Alg. 1): not the oracle, and not part of the GPU library.  Built with
gcc -O3 -fopenmp for the host it runs on.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hogwild.c")
_LIB = os.path.join(_HERE, "libhogwild.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.hogwild_threads.restype = C.c_int
        L.hogwild_threads.argtypes = []
        L.hogwild_train_level.restype = C.c_int64
        L.hogwild_train_level.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                          C.c_double, C.c_double, C.c_uint64]
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().hogwild_threads())


def train_level(rowptr, col, M, k, epochs, lr, lr_floor=1e-4, seed=1) -> int:
    """Trains M (float32 n x d, C-contiguous, in place); returns updates applied."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    assert M.dtype == np.float32 and M.flags.c_contiguous and M.shape[0] == len(rowptr) - 1
    return int(lib().hogwild_train_level(M.shape[0], rowptr.ctypes.data, col.ctypes.data, M.ctypes.data,
                                         M.shape[1], k, epochs, lr, lr_floor, seed))
