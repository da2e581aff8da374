"""CPU oracle for the blocked SpMV -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product path (``paper_2605_18515_gb300`` and its CUDA library)
never imports it, and the two share no code: the only common module is the seeded input
generator ``paper_2605_18515_gb300.inputs``, which holds none of the method's arithmetic.

Contents
  * ``spmv`` / ``spmv_rows`` / ``spmm``: the CSR SpMV of Sec. 2.2, Algorithm 1, with BLAS
    alpha/beta scaling, in plain C (``cb_oracle.c``, IEEE double, no FMA contraction).
  * ``dense_gemv_ld``: brute-force dense product in long double for tiny inputs.
  * ``oracle.blocked``: the preprocessing steps of Sec. 3 in the paper's order (2D tiling,
    the column-aggregation decision and aggregation, format selection, the coordinate
    byte of Sec. 3.2 and the thread-block load balance of Algorithm 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "cb_oracle.c")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def lib_path(mutant: int = 0) -> str:
    return os.path.join(_BUILD, "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile cb_oracle.c with gcc (mutant > 0 plants a known mistake, for tests)."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", *CFLAGS, f"-DORACLE_MUTANT={mutant}", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutant not in _libs:
            L = ctypes.CDLL(build(mutant))
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            L.oracle_spmv_csr.argtypes = [i64, i64, P, P, P, P, d, d, P, P, P]
            L.oracle_spmv_csr_rows.argtypes = [i64, P, P, P, P, P, d, d, P, P, P]
            L.oracle_spmm_csr.argtypes = [i64, i64, P, P, P, P, i64, d, d, P, i64, P, P]
            L.oracle_dense_gemv_ld.argtypes = [i64, i64, P, P, P]
            L.oracle_mutant_id.restype = ctypes.c_int
            for f in (L.oracle_spmv_csr, L.oracle_spmv_csr_rows, L.oracle_spmm_csr,
                      L.oracle_dense_gemv_ld):
                f.restype = None
            _libs[mutant] = L
        return _libs[mutant]


def _p(a):
    return None if a is None else a.ctypes.data


def _csr_arrays(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, col, val


def spmv(A, x, alpha=1.0, beta=0.0, y0=None, mutant: int = 0):
    """y = alpha*A*x + beta*y0 and s_i = sum_k |a_ik x_k|, both float64 arrays of length m."""
    rp, col, val = _csr_arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape[0] >= A.n
    y = np.empty(A.m, dtype=np.float64)
    s = np.empty(A.m, dtype=np.float64)
    if beta != 0.0:
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        assert y0.shape[0] >= A.m
    else:
        y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
    _lib(mutant).oracle_spmv_csr(A.m, A.n, _p(rp), _p(col), _p(val), _p(x), alpha, beta, _p(y0),
                                 _p(y), _p(s))
    return y, s


def spmv_rows(A, x, rows, alpha=1.0, beta=0.0, y0=None):
    """The product for the listed rows only: returns (y[rows], s[rows])."""
    rp, col, val = _csr_arrays(A)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(rows.size, dtype=np.float64)
    s = np.empty(rows.size, dtype=np.float64)
    if beta != 0.0:
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
    _lib().oracle_spmv_csr_rows(rows.size, _p(rows), _p(rp), _p(col), _p(val), _p(x), alpha, beta,
                                _p(y0 if beta != 0.0 else None), _p(y), _p(s))
    return y, s


def spmm(A, X, alpha=1.0, beta=0.0, Y0=None):
    """k right-hand sides: X (k, n) -> Y (k, m), S (k, m)."""
    rp, col, val = _csr_arrays(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    k = X.shape[0]
    Y = np.empty((k, A.m), dtype=np.float64)
    S = np.empty((k, A.m), dtype=np.float64)
    if beta != 0.0:
        Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    _lib().oracle_spmm_csr(A.m, k, _p(rp), _p(col), _p(val), _p(X), X.shape[1], alpha, beta,
                           _p(Y0 if beta != 0.0 else None), A.m, _p(Y), _p(S))
    return Y, S


def dense_gemv_ld(D, x):
    """Brute-force dense product (long double accumulation) for tiny matrices."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(D.shape[0], dtype=np.float64)
    _lib().oracle_dense_gemv_ld(D.shape[0], D.shape[1], _p(D), _p(x), _p(y))
    return y


def within_tolerance(y_gpu, y_ref, s, alpha=1.0, beta=0.0, y0=None, rtol=1e-12):
    """Per-row acceptance test |y - y_ref| <= rtol * (|alpha| s_i + |beta y0_i|); rows whose
    scale is 0 must match exactly. Returns (ok, worst normalised error)."""
    scale = abs(alpha) * s
    if beta != 0.0:
        scale = scale + np.abs(beta * y0)
    err = np.abs(np.asarray(y_gpu, dtype=np.float64) - y_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        norm = np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), np.where(err > 0, np.inf, 0.0))
    worst = float(norm.max()) if norm.size else 0.0
    return bool(np.all(norm <= rtol)), worst
