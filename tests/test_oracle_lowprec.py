"""Pins of the oracle's reduced-precision rounding (oracle/lowprec.py) against numpy's own
correctly rounded conversions and hand-derived cases, and the library analyser's stored
values against the oracle (host-only handles, no GPU)."""
import numpy as np
import pytest

from oracle import lowprec as L
from paper_2605_18515_gb300 import build, inputs as I


def edge_values():
    rng = np.random.default_rng(1)
    v = np.concatenate([
        rng.standard_normal(20000) * 10.0 ** rng.integers(-12, 12, 20000),
        rng.standard_normal(2000) * 1e-40, rng.standard_normal(2000) * 1e-6,   # subnormal ranges
        np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 1e300, -1e300, 5e-324,
                  3.4028234663852886e38, 3.4028235677973366e38, 2.0 ** -149, 2.0 ** -150,
                  1.5 * 2.0 ** -149, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26]),
    ])
    # exact ties of float32: 1 + (2j+1) 2^-24 lie halfway between two float32 neighbours
    ties32 = 1.0 + (2 * np.arange(50) + 1) * 2.0 ** -24
    ties16 = 1.0 + (2 * np.arange(50) + 1) * 2.0 ** -11
    return np.concatenate([v, ties32, -ties32, ties16, -ties16])


def test_f32_matches_numpy_cast():
    v = edge_values()
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32).astype(np.float64)
    got = L.round_to_format(v, "f32")
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_f16_matches_numpy_cast():
    v = edge_values()
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).astype(np.float64)
    got = L.round_to_format(v, "f16")
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_bf16_hand_cases():
    e = 2.0 ** -8     # half an ulp of 1 in bfloat16 (7 fraction bits)
    cases = {
        1.0 + e: 1.0,                             # tie -> even (1.0)
        1.0 + 3 * e: 1.0 + 4 * e,                 # tie -> even (1 + 2^-6)
        1.0 + e * 1.0000001: 1.0 + 2 * e,         # just above the tie
        -(1.0 + 3 * e): -(1.0 + 4 * e),
    }
    for v, want in cases.items():
        assert L.round_to_format(np.array([v]), "bf16")[0] == want
    # largest finite bfloat16: (2 - 2^-7) 2^127; halfway to 2^128 rounds to infinity
    big = (2.0 - 2.0 ** -7) * 2.0 ** 127
    assert L.round_to_format(np.array([big]), "bf16")[0] == big
    assert np.isinf(L.round_to_format(np.array([(2.0 - 2.0 ** -8) * 2.0 ** 127]), "bf16")[0])
    # smallest subnormal 2^-133; half of it ties to zero (even), 0.75 of it rounds up
    tiny = 2.0 ** -133
    assert L.round_to_format(np.array([tiny, tiny / 2, 0.75 * tiny]), "bf16").tolist() == [tiny, 0.0, tiny]
    # values representable in bfloat16 are unchanged
    r = np.random.default_rng(3).standard_normal(5000).astype(np.float32)
    b = (r.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    assert np.array_equal(L.round_to_format(b, "bf16"), b)


def test_bf16_is_within_half_an_ulp():
    """Every rounded value has 8 significant bits and lies within half a bfloat16 ulp of
    the input (the ulp taken in the binade of the input)."""
    v = np.random.default_rng(4).standard_normal(20000) * 100
    got = L.round_to_format(v, "bf16")
    f, _ = np.frexp(got)
    assert np.all(np.ldexp(f, 8) == np.rint(np.ldexp(f, 8)))     # 8 significant bits
    ulp = np.ldexp(1.0, np.frexp(np.abs(v))[1] - 8)
    assert np.all(np.abs(got - v) <= ulp / 2)


@pytest.fixture(scope="module")
def bd():
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
def test_analyser_stores_oracle_rounded_values(bd, fmt):
    A = I.random_csr(300, 280, 0.3, 21)
    rng = np.random.default_rng(7)
    A.val = A.val * 10.0 ** rng.integers(-9, 9, A.val.size)    # spread over the exponent range
    with bd.BlockedMatrix(A, device=-1, value_dtype=fmt) as M:
        rp, col, val = M.export_csr()
        st = M.stats()
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    ref = L.round_to_format(A.val, fmt)
    assert np.array_equal(val.view(np.uint64), ref.view(np.uint64))
    vs = {"f32": 4, "bf16": 2, "f16": 2}[fmt]
    assert st["value_dtype"] == {"f32": 1, "bf16": 2, "f16": 3}[fmt]
    assert st["algo_bytes_per_run"] >= A.nnz * (vs + 1)


def test_fp32_bound_catches_a_dropped_term():
    """The FP32 acceptance bound is tight enough that losing one product of a row fails."""
    import oracle
    A = I.random_csr(200, 200, 0.2, 9)
    x = I.vector_x(A.n, 3).astype(np.float32).astype(np.float64)
    y, s = oracle.spmv(A, x)
    bad = y.copy()
    r = int(np.argmax(np.diff(A.row_ptr)))
    k = A.row_ptr[r]
    bad[r] -= A.val[k] * x[A.col[k]]
    assert L.within_bound(y, y, s, L.fp32_bound(A))[0]
    assert not L.within_bound(bad, y, s, L.fp32_bound(A))[0]


def _fp32_orders(p):
    """Sums of the FP32 products p (float32 array) in five FP32 evaluation orders: left to
    right, right to left, a pairwise tree, 32 strided partial sums added by a halving tree
    (a warp's order), and one random permutation."""
    f = np.float32
    out = []
    for seq in (p, p[::-1], np.random.default_rng(p.size).permutation(p)):
        acc = f(0)
        for v in seq:
            acc = f(acc + v)
        out.append(acc)
    def tree(v):
        v = list(v) or [f(0)]
        while len(v) > 1:
            v = [f(v[i] + v[i + 1]) if i + 1 < len(v) else v[i] for i in range(0, len(v), 2)]
        return v[0]
    out.append(tree(p))
    lanes = [f(0)] * 32
    for i, v in enumerate(p):
        lanes[i % 32] = f(lanes[i % 32] + v)
    out.append(tree(lanes))
    return out


def test_fp32_bound_holds_for_every_evaluation_order():
    """Soundness of the acceptance bound (Higham, Sec. 3.1): a row of k FP32 products summed in
    FP32 in any order, then scaled by alpha and updated with beta y0 in FP32, stays within
    fp32_bound's gamma_{k + 10} times sum |a x| of the exact result (exact products and a
    correctly rounded sum, math.fsum). Rows of 1..400 entries mixing signs and 12 decades."""
    import math
    from paper_2605_18515_gb300.inputs import CSR
    rng = np.random.default_rng(21)
    f = np.float32
    worst = 0.0
    for trial in range(60):
        k = int(rng.integers(1, 401))
        a = (rng.standard_normal(k) * 10.0 ** rng.integers(-6, 6, k)).astype(f)
        x = rng.uniform(-1, 1, k).astype(f)
        alpha, beta, y0 = (f(1), f(0), f(0)) if trial % 2 else (f(-0.7), f(1.3), f(rng.standard_normal()))
        A = CSR(1, k, np.array([0, k], np.int64), np.arange(k, dtype=np.int32), a.astype(np.float64))
        g = L.fp32_bound(A)[0]
        exact_terms = [float(ai) * float(xi) for ai, xi in zip(a, x)]   # exact in FP64 (24 + 24 bits)
        dot = math.fsum(exact_terms)
        exact = float(alpha) * dot + float(beta) * float(y0)
        scale = abs(float(alpha)) * math.fsum(abs(t) for t in exact_terms) + abs(float(beta) * float(y0))
        for sfp in _fp32_orders((a * x).astype(f)):
            y = f(f(alpha * sfp) + f(beta * y0))
            err = abs(float(y) - exact)
            assert err <= g * scale, (trial, k, err / scale, g)
            worst = max(worst, err / scale / g)
    assert worst > 0.0


def test_fp32_bound_is_nearly_attained():
    """Tightness: the bound is not loose by more than a small factor. A row holding 1 and
    then k - 1 entries of 2^-24 (x = 1) summed left to right in FP32 stays at 1 (each
    1 + 2^-24 is a tie that rounds to even), an error of (k - 1) 2^-24 against a scale of
    1 + (k - 1) 2^-24: that is (k - 1) / (k + 10) of gamma_{k + 10}, within it and above 0.8
    of it for k = 128. A unit roundoff of 2^-23 in the bound (twice too loose) fails here."""
    from paper_2605_18515_gb300.inputs import CSR
    f = np.float32
    k = 128
    a = np.concatenate([[1.0], np.full(k - 1, 2.0 ** -24)])
    A = CSR(1, k, np.array([0, k], np.int64), np.arange(k, dtype=np.int32), a)
    acc = f(0)
    for v in a.astype(f):
        acc = f(acc + v)
    assert acc == f(1)
    exact = 1.0 + (k - 1) * 2.0 ** -24
    ratio = abs(float(acc) - exact) / exact / L.fp32_bound(A)[0]
    assert 0.8 < ratio <= 1.0, ratio
