"""Reduced-precision value storage for the oracle -- test infrastructure only (imported by
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` only).

The paper names a mixed-precision form of the method (Sec. 2.2) but fixes none of its
arithmetic. The reading tested here:
  * each FP64 matrix value is rounded to the nearest number of the storage format
    (binary32, bfloat16 or binary16), ties to even, directly from FP64; magnitudes past
    the largest finite number become infinities; below the smallest normal number the
    format's subnormal quantum applies;
  * x, y, alpha and beta are FP32 and every product and sum is formed in FP32.
The oracle's reference result is the exact product of the stored (rounded) values and the
FP32 x, formed by the FP64 CSR oracle (whose own rounding is ~1e-16 relative, far below
the FP32 bound); ``fp32_bound`` gives the classical bound on any FP32 evaluation order
(Higham, "Accuracy and Stability of Numerical Algorithms", Sec. 3.1: a sum of k products
in any order has error at most gamma_k times the sum of absolute values, gamma_k =
k u / (1 - k u)).

Pins (tests/test_oracle_lowprec.py): ``round_to_format`` equals numpy's own correctly
rounded float64 -> float32 and float64 -> float16 conversions on random, tie, subnormal
and overflow inputs, and hand-derived bfloat16 cases. ``fp32_bound`` holds for five FP32
evaluation orders of random rows against the exact sum (math.fsum of exact products), is
attained to within 0.8 by a row of ties that left-to-right FP32 summation rounds away, and
rejects a result with one product dropped.
"""
from __future__ import annotations

import numpy as np

# significand bits (implicit bit included), smallest normal exponent, largest exponent
FORMATS = {"f32": (24, -126, 127), "bf16": (8, -126, 127), "f16": (11, -14, 15)}
# unit roundoff of each storage format and of the FP32 arithmetic
UNIT_ROUNDOFF = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
U32 = 2.0 ** -24


def round_to_format(v, fmt: str) -> np.ndarray:
    """v (float64 array) rounded to nearest, ties to even, in format fmt; returned as
    float64 (exact)."""
    p, emin, emax = FORMATS[fmt]
    v = np.asarray(v, dtype=np.float64)
    out = v.copy()
    fin = np.isfinite(v) & (v != 0.0)
    w = v[fin]
    _, e = np.frexp(w)               # w = f * 2**e with 0.5 <= |f| < 1
    E = np.maximum(e - 1, emin)      # floor(log2|w|), clamped at the subnormal range
    q = E - (p - 1)                  # exponent of the quantum (one unit in the last place)
    with np.errstate(over="ignore", invalid="ignore"):
        r = np.rint(np.ldexp(w, -q))     # nearest integer, ties to even
        res = np.ldexp(r, q)
    largest = np.ldexp(2.0 - 2.0 ** (1 - p), emax)
    too_big = (e - 1 > emax) | ~np.isfinite(res) | (np.abs(res) > largest)
    res = np.where(too_big, np.copysign(np.inf, w), res)
    out[fin] = res
    return out


def stored_matrix(A, fmt: str):
    """A copy of the CSR matrix A with its values replaced by the stored (rounded) values."""
    return type(A)(A.m, A.n, A.row_ptr, A.col, round_to_format(A.val, fmt))


def fp32_bound(A, k_extra: int = 10) -> np.ndarray:
    """Per-row factor gamma_{k_i + k_extra} for FP32 arithmetic, k_i = stored entries of
    row i; k_extra covers the merges of partial sums, the alpha scaling and the beta
    update."""
    k = np.diff(np.asarray(A.row_ptr, dtype=np.int64)).astype(np.float64) + k_extra
    return k * U32 / (1.0 - k * U32)


def within_bound(y_gpu, y_ref, scale, factor):
    """|y_gpu - y_ref| <= factor * scale per row (rows with scale 0 must match exactly).
    Returns (ok, worst of |error| / scale)."""
    err = np.abs(np.asarray(y_gpu, dtype=np.float64) - np.asarray(y_ref, dtype=np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        norm = np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), np.where(err > 0, np.inf, 0.0))
    ok = bool(np.all(np.where(scale > 0, err <= factor * scale, err == 0)))
    return ok, (float(norm.max()) if norm.size else 0.0)
