"""Builds and loads the oracle's plain C part (kmeans_exact.c) with gcc.

Test infrastructure only. Compiled without fused multiply-add
(-ffp-contract=off) so that the dense FP64 sums are plain IEEE additions and
multiplications in the order the source writes them. Built with OpenMP when
gcc supports it (only the Lloyd assignment step uses threads, and its results
do not depend on their number), else without.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmeans_exact.c")
_LIB = os.path.join(_HERE, "_oracle_c.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile kmeans_exact.c into _oracle_c.so (next to the source)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:-1] + ["-fopenmp", "-lm"], capture_output=True).returncode:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _handle
    with _lock:
        if _handle is None:
            _handle = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            _handle.oracle_set_threads.restype = ctypes.c_int
            _handle.oracle_set_threads.argtypes = [ctypes.c_int]
            _handle.oracle_splitmix64.restype = u64
            _handle.oracle_splitmix64.argtypes = [u64, i64]
            _handle.oracle_u53.restype = ctypes.c_double
            _handle.oracle_u53.argtypes = [u64, i64]
            _handle.oracle_kmeanspp_binary.restype = ctypes.c_int
            _handle.oracle_kmeanspp_binary.argtypes = [i64, i64, P, P, P, P, i32, u64, P]
            _handle.oracle_lloyd_binary.restype = ctypes.c_int
            _handle.oracle_lloyd_binary.argtypes = [i64, i64, P, P, P, P, i32, P, i32, P, P]
            _handle.oracle_kmeanspp_dense.restype = ctypes.c_int
            _handle.oracle_kmeanspp_dense.argtypes = [i64, i64, P, i32, u64, P]
            _handle.oracle_lloyd_dense.restype = ctypes.c_int
            _handle.oracle_lloyd_dense.argtypes = [i64, i64, P, i32, P, i32, P, P]
        return _handle
