"""CSR x dense block product for the oracle (FP64).

``csr_spmm(row_ptr, col, val, X)`` returns Y = H X for H in CSR form.  It is a
library primitive of the oracle: SciPy's CSR product for small matrices, and a
plain C loop (one row after another, entries in stored order, OpenMP over rows;
``spmm.c``) for large ones so that a 4e8-nonzero product takes seconds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle_spmm.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "spmm.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", _SO + ".tmp", src], check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_csr_spmm.restype = None
        lib.oracle_csr_spmm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_set_threads.restype = None
        lib.oracle_set_threads.argtypes = [ctypes.c_int32]
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def csr_spmm(row_ptr: np.ndarray, col: np.ndarray, val: np.ndarray, X: np.ndarray, use_c: bool | None = None) -> np.ndarray:
    """Y = H X with H given by (row_ptr, col, val); X is n x k (any layout).

    use_c: force (True) or forbid (False) the C loop; default: C for >= 5e6 nonzeros.
    """
    n = row_ptr.shape[0] - 1
    X = np.ascontiguousarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    k = X.shape[1]
    if k > 64:
        return np.hstack([csr_spmm(row_ptr, col, val, X[:, c:c + 64], use_c) for c in range(0, k, 64)])
    if use_c is None:
        use_c = col.shape[0] >= 5_000_000
    if not use_c:
        H = sp.csr_matrix((val, col, row_ptr), shape=(n, X.shape[0]))
        Y = np.asarray(H @ X)
    else:
        lib = _load()
        Y = np.empty((n, k), dtype=np.float64)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cc = np.ascontiguousarray(col, dtype=np.int32)
        vv = np.ascontiguousarray(val, dtype=np.float64)
        lib.oracle_csr_spmm(n, k, rp.ctypes.data, cc.ctypes.data, vv.ctypes.data, X.ctypes.data, Y.ctypes.data)
    return Y[:, 0] if squeeze else Y
