"""The oracle's CSR product on several host threads — TEST INFRASTRUCTURE ONLY.

`spmv_threads(A, x, threads)` computes y = A x like `oracle.spmv` (one pass
over the rows of the assembled float64 matrix, entries in stored order), in
the plain C loop of csr_spmv.c with the rows split across `threads` threads.
It exists to time the oracle on all host cores for the benchmark's CPU
baseline; `build()` compiles it (gcc, OpenMP) next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csr_spmv.c")
_LIB = os.path.join(_HERE, "libcsr_spmv.so")
_lib = None


def build() -> str:
    """Compile csr_spmv.c into libcsr_spmv.so (no-op when up to date)."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _LIB]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed:\n{r.stdout}\n{r.stderr}")
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise ImportError(f"{_LIB} not built; call oracle.cpu_spmv.build()")
        lib = ctypes.CDLL(_LIB)
        lib.oracle_csr_spmv.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
        lib.oracle_csr_spmv.restype = None
        _lib = lib
    return _lib


def host_cores() -> int:
    """Cores this process may run on (the affinity mask, else os.cpu_count())."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class CsrOperands:
    """A's arrays in the C loop's types (int64 row pointers, int32 columns)."""

    def __init__(self, A: sp.csr_matrix):
        A = A.tocsr()
        self.n_rows = A.shape[0]
        self.indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.data = np.ascontiguousarray(A.data, dtype=np.float64)


def spmv_threads(ops: CsrOperands, x: np.ndarray, threads: int, y: np.ndarray | None = None) -> np.ndarray:
    """y = A x on `threads` threads (A given as CsrOperands)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    if y is None:
        y = np.empty(ops.n_rows, dtype=np.float64)
    lib.oracle_csr_spmv(ops.n_rows, ops.indptr.ctypes.data, ops.indices.ctypes.data, ops.data.ctypes.data,
                        x.ctypes.data, y.ctypes.data, int(threads))
    return y
