"""Pins for the CPU oracle's SpMV (Sec. 2.2, Algorithm 1) against facts that do not come
from the oracle itself: exact products of identity / diagonal / permutation matrices,
exact rational arithmetic on tiny inputs with the textbook rounding bound, closed-form
Laplacian row sums and eigenpairs, BLAS alpha/beta semantics, and planted mistakes that
the pins must catch."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_18515_gb300 import inputs as I

U = 2.0 ** -53


def diag_csr(d):
    n = d.size
    return I.CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d.astype(np.float64))


def perm_csr(p, vals=None):
    n = p.size
    v = np.ones(n) if vals is None else vals
    return I.CSR(n, n, np.arange(n + 1, dtype=np.int64), p.astype(np.int32), v.astype(np.float64))


# ---- pins written as functions of an spmv callable so that mutants can be run through them
def pin_identity(spmv):
    n = 300
    x = I.vector_x(n, 11)
    y, _ = spmv(diag_csr(np.ones(n)), x)
    return np.array_equal(y, x)


def pin_diagonal(spmv):
    n = 257
    d = I.uniform_pm1(5, 7, n)
    x = I.vector_x(n, 12)
    y, _ = spmv(diag_csr(d), x)
    return np.array_equal(y, d * x)          # one correctly rounded product per row


def pin_permutation(spmv):
    n = 200
    p = np.argsort(I.uniform01(3, 9, n))
    x = I.vector_x(n, 13)
    y, _ = spmv(perm_csr(p), x)               # row i holds a single 1 at column p[i]
    return np.array_equal(y, x[p])


def pin_laplacian_ones(spmv):
    g = 64
    A = I.laplacian2d(g)
    y, _ = spmv(A, np.ones(A.n))
    i, j = np.divmod(np.arange(g * g), g)
    nb = (i > 0).astype(int) + (i < g - 1) + (j > 0) + (j < g - 1)
    return np.array_equal(y, 4.0 - nb)        # 0 inside, 1 on edges, 2 at corners


def pin_laplacian_eigen(spmv):
    g = 64
    A = I.laplacian2d(g)
    ok = True
    for p, q in ((1, 1), (3, 7), (64, 1), (32, 33)):
        ii, jj = np.divmod(np.arange(g * g), g)
        v = np.sin(np.pi * p * (ii + 1) / (g + 1)) * np.sin(np.pi * q * (jj + 1) / (g + 1))
        lam = 4 - 2 * np.cos(np.pi * p / (g + 1)) - 2 * np.cos(np.pi * q / (g + 1))
        y, s = spmv(A, v)
        ok &= bool(np.all(np.abs(y - lam * v) <= 1e-12 * (s + np.abs(lam * v))))
    return ok


def pin_alpha_beta(spmv):
    A = I.random_csr(40, 30, 0.3, 21)
    x = I.vector_x(30, 22)
    y0 = I.uniform_pm1(23, 4, 40)
    y1, _ = spmv(A, x, 1.0, 0.0)
    y2, _ = spmv(A, x, 2.0, 0.0)
    y3, _ = spmv(A, x, 0.0, 1.0, y0)
    y4, _ = spmv(A, x, 2.0, -0.5, y0)
    return (np.array_equal(y2, 2.0 * y1) and np.array_equal(y3, y0)
            and np.array_equal(y4, 2.0 * y1 + (-0.5) * y0))


def pin_beta_zero_ignores_y(spmv):
    A = I.random_csr(33, 33, 0.2, 31)
    x = I.vector_x(33, 32)
    y0 = np.full(33, np.nan)
    y, _ = spmv(A, x, 1.0, 0.0, y0)
    yref, _ = spmv(A, x)
    return np.array_equal(y, yref) and not np.isnan(y).any()


def pin_exact_rational(spmv):
    ok = True
    for seed, (m, n, dens) in enumerate(((17, 23, 0.3), (40, 40, 0.9), (64, 5, 0.5), (3, 64, 1.0))):
        A = I.random_csr(m, n, dens, 100 + seed)
        x = I.vector_x(n, 200 + seed)
        y, s = spmv(A, x)
        for r in range(m):
            lo, hi = A.row_ptr[r], A.row_ptr[r + 1]
            exact = sum((Fraction(float(A.val[k])) * Fraction(float(x[A.col[k]])) for k in range(lo, hi)), Fraction(0))
            L = hi - lo
            gamma = L * U / (1 - L * U) if L else 0.0
            bound = gamma * sum(abs(float(A.val[k]) * float(x[A.col[k]])) for k in range(lo, hi)) * (1 + 1e-12)
            ok &= abs(Fraction(float(y[r])) - exact) <= Fraction(bound)
            if L == 0:
                ok &= y[r] == 0.0
    return ok


def pin_dense_bruteforce(spmv):
    A = I.random_csr(48, 48, 0.6, 41)
    x = I.vector_x(48, 42)
    D = np.zeros((48, 48))
    D[A.rows(), A.col] = A.val
    y, s = spmv(A, x)
    return bool(np.all(np.abs(y - oracle.dense_gemv_ld(D, x)) <= 48 * U * s + 1e-300))


def pin_nonsymmetric_transpose(spmv):
    # a strictly upper bidiagonal matrix: (Ax)_i = x_{i+1}; its transpose gives x_{i-1}
    n = 50
    rp = np.concatenate([np.arange(n, dtype=np.int64), [n - 1]])
    A = I.CSR(n, n, rp, np.arange(1, n, dtype=np.int32), np.ones(n - 1))
    x = I.vector_x(n, 43)
    y, _ = spmv(A, x)
    return np.array_equal(y[:-1], x[1:]) and y[-1] == 0.0


PINS = [pin_identity, pin_diagonal, pin_permutation, pin_laplacian_ones, pin_laplacian_eigen,
        pin_alpha_beta, pin_beta_zero_ignores_y, pin_exact_rational, pin_dense_bruteforce,
        pin_nonsymmetric_transpose]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    assert pin(oracle.spmv)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_pins_catch_planted_mistakes(mutant):
    """Each planted mistake in the oracle (see cb_oracle.c) must fail at least one pin."""
    def spmv(A, x, alpha=1.0, beta=0.0, y0=None):
        return oracle.spmv(A, x, alpha, beta, y0, mutant=mutant)
    failed = []
    for pin in PINS:
        try:
            ok = pin(spmv)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} passed every pin"


def test_laplacian3d_closed_form():
    g = 12
    A = I.laplacian3d(g)
    idx = np.arange(g ** 3)
    i, j, k = idx // (g * g), (idx // g) % g, idx % g
    y, _ = oracle.spmv(A, np.ones(A.n))
    nb = sum(((a > 0).astype(int) + (a < g - 1)) for a in (i, j, k))
    assert np.array_equal(y, 6.0 - nb)
    p, q, r = 2, 5, 11
    v = (np.sin(np.pi * p * (i + 1) / (g + 1)) * np.sin(np.pi * q * (j + 1) / (g + 1))
         * np.sin(np.pi * r * (k + 1) / (g + 1)))
    lam = 6 - 2 * sum(np.cos(np.pi * t / (g + 1)) for t in (p, q, r))
    y, s = oracle.spmv(A, v)
    assert np.all(np.abs(y - lam * v) <= 1e-12 * (s + np.abs(lam * v)))


def test_rows_and_multi_rhs_agree_with_full():
    A = I.random_csr(70, 50, 0.25, 51)
    X = I.vector_x(50, 52, k=3)
    Y0 = I.uniform_pm1(53, 4, 3 * 70).reshape(3, 70)
    Y, S = oracle.spmm(A, X, 1.5, 0.25, Y0)
    for j in range(3):
        y, s = oracle.spmv(A, X[j], 1.5, 0.25, Y0[j])
        assert np.array_equal(Y[j], y) and np.array_equal(S[j], s)
    rows = np.array([0, 69, 7, 7, 33])
    yr, sr = oracle.spmv_rows(A, X[1], rows, 1.5, 0.25, Y0[1])
    assert np.array_equal(yr, Y[1][rows]) and np.array_equal(sr, S[1][rows])


def test_tolerance_helper():
    y = np.array([1.0, 0.0, 2.0])
    ok, worst = oracle.within_tolerance(y + np.array([1e-13, 0, 0]), y, np.array([1.0, 0.0, 1.0]))
    assert ok and worst == pytest.approx(1e-13, rel=1e-3)
    ok, worst = oracle.within_tolerance(y + np.array([0, 1e-300, 0]), y, np.array([1.0, 0.0, 1.0]))
    assert not ok
