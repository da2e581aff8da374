"""GPU parity of the blocked SpMV against the CPU oracle, through the C ABI.

Acceptance (per row): |y_gpu - y_oracle| <= 1e-12 * (|alpha| * sum_k |a_ik x_k| + |beta y0_i|),
rows whose scale is zero must match exactly. Cases span several tiles and ragged tails,
every sub-block format and threshold boundary, aggregation on and off, split block rows,
empty inputs, BLAS alpha/beta semantics, and the full-size configurations (sampled rows).
"""
import numpy as np
import pytest

import oracle
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def gpu_spmv(env, A, x, alpha=1.0, beta=0.0, y0=None, reps=1, **opts):
    bd, torch = env
    with bd.BlockedMatrix(A, **opts) as M:
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        outs = []
        for _ in range(reps):
            yd = torch.from_numpy(np.array(y0 if y0 is not None else np.zeros(A.m), dtype=np.float64)).cuda()
            M.run(xd, yd, alpha, beta)
            outs.append(yd.cpu().numpy())
        torch.cuda.synchronize()
        M.check_device()
        st = M.stats()
    return (outs if reps > 1 else outs[0]), st


def check(A, x, y, alpha=1.0, beta=0.0, y0=None):
    yref, s = oracle.spmv(A, x, alpha, beta, y0)
    ok, worst = oracle.within_tolerance(y, yref, s, alpha, beta, y0, RTOL)
    assert ok, f"worst normalised error {worst:.3e}"
    return worst


SMALL = {
    "laplace2d_64": lambda: I.laplacian2d(64),
    "laplace3d_10": lambda: I.laplacian3d(10),
    "ragged_203x157": lambda: I.random_csr(203, 157, 0.07, 5),
    "dense_70x45": lambda: I.random_csr(70, 45, 0.85, 6),
    "mixed_333x517": lambda: I.random_csr(333, 517, 0.2, 11),
    "rmat12": lambda: I.rmat(12, 16, seed=4),
    "fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
    "one_row": lambda: I.random_csr(1, 3000, 0.5, 7),
    "one_col": lambda: I.random_csr(3000, 1, 0.5, 8),
    "tall_skinny": lambda: I.random_csr(5000, 17, 0.3, 12),
}


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("col_agg", [-1, 0, 1])
@pytest.mark.parametrize("layout", ["lanes", "records"])
def test_parity_small(env, name, col_agg, layout):
    A = SMALL[name]()
    x = I.vector_x(A.n, 100)
    y, st = gpu_spmv(env, A, x, col_agg=col_agg, record_layout=layout == "records")
    assert st["lane_layout"] == (layout == "lanes")
    check(A, x, y)


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.5, 0.0), (1.0, 1.0), (-0.5, 0.25), (0.0, 2.0), (0.0, 0.0)])
def test_alpha_beta(env, alpha, beta):
    A = I.random_csr(301, 260, 0.1, 21)
    x = I.vector_x(A.n, 22)
    y0 = I.uniform_pm1(23, I.TAG_Y, A.m)
    y, _ = gpu_spmv(env, A, x, alpha, beta, y0)
    check(A, x, y, alpha, beta, y0)


def test_beta_zero_ignores_nan_in_y(env):
    A = I.random_csr(100, 100, 0.2, 31)
    x = I.vector_x(A.n, 32)
    y, _ = gpu_spmv(env, A, x, 1.0, 0.0, np.full(A.m, np.nan))
    assert not np.isnan(y).any()
    check(A, x, y)


def test_exact_special_matrices(env):
    n = 1000
    x = I.vector_x(n, 41)
    d = I.uniform_pm1(42, 7, n)
    eye = I.CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    assert np.array_equal(gpu_spmv(env, eye, x)[0], x)
    diag = I.CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d)
    assert np.array_equal(gpu_spmv(env, diag, x)[0], d * x)
    p = np.argsort(I.uniform01(43, 9, n))
    perm = I.CSR(n, n, np.arange(n + 1, dtype=np.int64), p.astype(np.int32), np.ones(n))
    for agg in (0, 1):
        assert np.array_equal(gpu_spmv(env, perm, x, col_agg=agg)[0], x[p])


def test_laplacian_closed_forms(env):
    g = 64
    A = I.laplacian2d(g)
    i, j = np.divmod(np.arange(g * g), g)
    nb = (i > 0).astype(int) + (i < g - 1) + (j > 0) + (j < g - 1)
    assert np.array_equal(gpu_spmv(env, A, np.ones(A.n))[0], 4.0 - nb)
    p, q = 5, 9
    v = np.sin(np.pi * p * (i + 1) / (g + 1)) * np.sin(np.pi * q * (j + 1) / (g + 1))
    lam = 4 - 2 * np.cos(np.pi * p / (g + 1)) - 2 * np.cos(np.pi * q / (g + 1))
    y, _ = gpu_spmv(env, A, v)
    _, s = oracle.spmv(A, v)
    assert np.all(np.abs(y - lam * v) <= 1e-12 * (s + np.abs(lam * v)))


@pytest.mark.parametrize("k", [1, 31, 32, 128, 129, 256])
def test_format_boundaries(env, k):
    # 40 sub-blocks each holding k entries: exercises COO / CSR / Dense at the thresholds
    idx = np.arange(k)
    r, c = [], []
    for b in range(40):
        r.append(16 * (b // 8) + idx // 16)
        c.append(16 * (b % 8) + ((idx % 16) + b) % 16)
    A = I.csr_from_coo(80, 128, np.concatenate(r), np.concatenate(c), I.uniform_pm1(3, 2, 40 * k))
    x = I.vector_x(A.n, 50)
    for agg in (0, 1):
        for rec in (False, True):
            y, st = gpu_spmv(env, A, x, col_agg=agg, record_layout=rec)
            check(A, x, y)


def test_empty_inputs(env):
    bd, torch = env
    for m, n in ((37, 0), (37, 50), (1, 1)):
        A = I.CSR(m, n, np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
        x = I.vector_x(max(n, 1), 1)[:n] if n else np.zeros(0)
        y0 = I.uniform_pm1(5, 4, m)
        with bd.BlockedMatrix(A) as M:
            xd = torch.zeros(max(n, 1), dtype=torch.float64, device="cuda")
            yd = torch.from_numpy(y0.copy()).cuda()
            M.run(xd, yd, 1.0, 0.5)
            assert np.array_equal(yd.cpu().numpy(), 0.5 * y0)
            M.run(xd, yd, 1.0, 0.0)
            assert np.array_equal(yd.cpu().numpy(), np.zeros(m))
    A = I.CSR(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    with bd.BlockedMatrix(A) as M:
        M.run(torch.zeros(5, dtype=torch.float64, device="cuda"), torch.zeros(1, dtype=torch.float64, device="cuda"))


def heavy_rows_matrix():
    # block rows far above one unit's budget (split into parts) next to sparse ones
    rng_r, rng_c = [], []
    for b, cols in ((0, 9000), (3, 2500), (7, 40000)):
        rr = np.repeat(np.arange(16 * b, 16 * b + 16), cols // 16)
        cc = (np.arange(rr.size) * 7919) % 50000
        rng_r.append(rr); rng_c.append(cc)
    sp = I.random_csr(400, 50000, 0.0005, 77)
    rng_r.append(sp.rows()); rng_c.append(sp.col)
    r = np.concatenate(rng_r); c = np.concatenate(rng_c)
    key = np.unique(r * 50000 + c)
    return I.csr_from_coo(400, 50000, key // 50000, key % 50000, I.uniform_pm1(8, 2, key.size),
                          sum_duplicates=False)


@pytest.mark.parametrize("layout", ["lanes", "records"])
def test_split_block_rows_and_determinism(env, layout):
    A = heavy_rows_matrix()
    x = I.vector_x(A.n, 60)
    ys, st = gpu_spmv(env, A, x, 1.5, 0.0, reps=3, record_layout=layout == "records")
    assert st["n_split_rows"] >= 3
    for y in ys:
        check(A, x, y, 1.5)
    assert all(np.array_equal(ys[0], y) for y in ys[1:])    # no scheduling dependence


def long_row_unit_matrix():
    # one block row of 512 columns (32 sub-blocks: one lane-stream unit) whose row 3 is full
    # (a row across every lane run: the segmented-scan carry path) and whose other rows hold
    # 0, 1 or a few entries; plus a second block row with empty rows between short ones
    r, c = [np.full(512, 3)], [np.arange(512)]
    for row in (0, 1, 7, 15):
        cols = np.arange(row, 512, 37 + row)
        r.append(np.full(cols.size, row)); c.append(cols)
    r.append(np.array([17, 17, 30])); c.append(np.array([0, 500, 250]))
    r, c = np.concatenate(r), np.concatenate(c)
    return I.csr_from_coo(32, 512, r, c, I.uniform_pm1(19, 2, r.size))


def test_row_across_all_lanes(env):
    bd, torch = env
    A = long_row_unit_matrix()
    x = I.vector_x(A.n, 61)
    y0 = I.uniform_pm1(62, I.TAG_Y, A.m)
    for agg in (0, 1):
        y, st = gpu_spmv(env, A, x, 0.75, 0.5, y0, col_agg=agg)
        assert st["lane_layout"] == 1
        check(A, x, y, 0.75, 0.5, y0)
    with bd.BlockedMatrix(A) as M:
        for k in (2, 4, 7):
            X = np.stack([I.vector_x(A.n, 70 + j) for j in range(k)])
            Yd = torch.zeros((k, A.m), dtype=torch.float64, device="cuda")
            M.run_multi(torch.from_numpy(X).cuda(), Yd, 1.0, 0.0)
            Y = Yd.cpu().numpy()
            for j in range(k):
                check(A, X[j], Y[j])


@pytest.mark.parametrize("unit_work", [64, 300, 4000])
def test_unit_sizes(env, unit_work):
    A = I.random_csr(900, 700, 0.05, 13)
    x = I.vector_x(A.n, 14)
    y, st = gpu_spmv(env, A, x, unit_work=unit_work)
    check(A, x, y)


def test_small_matrix_units_spread_over_the_sms(env):
    """With fewer default lane units (2,048 entries) than CTAs the analysis shrinks the unit
    to max(256, largest block row, nnz / CTAs) entries: the 64x64 Laplacian (20,224
    entries, block rows of 80) gets one unit of ~256 entries per CTA instead of 37,
    and the product still matches the oracle; an explicit unit_work is kept as given (37
    units of at most 7 block rows)."""
    bd, torch = env
    A = I.laplacian2d(64)
    x = I.vector_x(A.n, 19)
    y, st = gpu_spmv(env, A, x)
    assert st["lane_layout"] == 1 and st["n_workers"] >= 100
    assert st["n_units"] >= 64 and st["n_split_units"] == 0
    check(A, x, y)
    y2, st2 = gpu_spmv(env, A, x, unit_work=2048)
    assert st2["n_units"] == 37 < st["n_units"]
    check(A, x, y2)


def test_load_balance_toggle_same_result(env):
    A = I.rmat(13, 16, seed=5)
    x = I.vector_x(A.n, 15)
    y1, _ = gpu_spmv(env, A, x, load_balance=True)
    y0, _ = gpu_spmv(env, A, x, load_balance=False)
    check(A, x, y1)
    assert np.array_equal(y0, y1)


def test_run_host_matches_device_path(env):
    bd, torch = env
    A = I.random_csr(500, 450, 0.05, 16)
    x = I.vector_x(A.n, 17)
    y0 = I.uniform_pm1(18, I.TAG_Y, A.m)
    with bd.BlockedMatrix(A) as M:
        yh = M.run_host(x, y0.copy(), 0.5, -1.0)
        yd = torch.from_numpy(y0.copy()).cuda()
        M.run(torch.from_numpy(x).cuda(), yd, 0.5, -1.0)
        assert np.array_equal(yh, yd.cpu().numpy())
    check(A, x, yh, 0.5, -1.0, y0)


def test_device_roundtrip(env):
    bd, _ = env
    A = I.rmat(12, 16, seed=8)
    with bd.BlockedMatrix(A) as M:
        rp, col, val = M.export_csr()
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    assert np.array_equal(val.view(np.uint64), A.val.view(np.uint64))


# ---- full-size configurations: every row checked for the FEM matrix is too slow for the
# pure oracle loop in a test, so a fixed sample of rows (first, last, hub rows and a
# seeded random set) is compared one by one; the whole vector is compared through
# properties that hold at any size (x = 1 row sums of the same matrix, determinism).
def sampled_rows(m, seed, k=20000, extra=()):
    rows = np.unique(np.concatenate([np.arange(min(m, 64)), np.arange(max(0, m - 64), m),
                                     (I.uniform01(seed, 9, k) * m).astype(np.int64), np.asarray(extra, np.int64)]))
    return rows[(rows >= 0) & (rows < m)]


@pytest.mark.slow
@pytest.mark.parametrize("name", ["fem3x3_band_1m", "rmat_s21"])
def test_full_size_configs(env, name):
    bd, torch = env
    A, x = I.config_matrix(name)
    deg = np.diff(A.row_ptr)
    rows = sampled_rows(A.m, 5, extra=np.argsort(deg)[-200:])
    with bd.BlockedMatrix(A) as M:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty(A.m, dtype=torch.float64, device="cuda")
        M.run(xd, yd)
        y1 = yd.cpu().numpy()
        M.run(xd, yd)
        y2 = yd.cpu().numpy()
        ones = torch.ones(A.n, dtype=torch.float64, device="cuda")
        M.run(ones, yd)
        y_ones = yd.cpu().numpy()
        M.check_device()
    assert np.array_equal(y1, y2)
    yref, s = oracle.spmv_rows(A, x, rows)
    ok, worst = oracle.within_tolerance(y1[rows], yref, s, rtol=RTOL)
    assert ok, f"{name}: worst normalised error {worst:.3e}"
    # x = 1: row sums of the stored values, checked on every row against the oracle scale
    yref1, s1 = oracle.spmv_rows(A, np.ones(A.n), rows)
    assert oracle.within_tolerance(y_ones[rows], yref1, s1, rtol=RTOL)[0]
    r = A.rows()
    absrow = np.bincount(r, weights=np.abs(A.val), minlength=A.m)
    rowsum = np.bincount(r, weights=A.val, minlength=A.m)
    assert np.all(np.abs(y_ones - rowsum) <= 1e-12 * absrow)


@pytest.mark.parametrize("kind", ["long_entry_unit", "short_entry_unit"])
def test_single_entry_units_with_and_without_direct_descriptors(env, kind):
    """A single-entry unit of 540 chunks keeps 16-bit descriptors (tile bases and coordinate
    bytes); one of 320 chunks carries direct descriptors. Both against the oracle, FP64,
    alpha/beta, and with several vectors per pass."""
    bd, torch = env
    # 540 entries (11 rows of two per tile), or 320 (every row one per tile)
    A = I.isolated_entries_block_row(rows_with_two=11 if kind == "long_entry_unit" else 0)
    x = I.vector_x(A.n, 41)
    y0 = I.uniform_pm1(42, I.TAG_Y, A.m)
    y, st = gpu_spmv(env, A, x, 1.5, -0.5, y0, col_agg=0, record_layout=True)
    assert st["n_entry_mode_units"] == 1
    assert st["n_direct_units"] == (0 if kind == "long_entry_unit" else 1)
    check(A, x, y, 1.5, -0.5, y0)
    y, st = gpu_spmv(env, A, x, 1.5, -0.5, y0, col_agg=0)
    assert st["lane_layout"] == 1
    check(A, x, y, 1.5, -0.5, y0)
    with bd.BlockedMatrix(A, col_agg=0, record_layout=True) as M:
        X = np.stack([I.vector_x(A.n, 50 + j) for j in range(7)])
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros((7, A.m), dtype=torch.float64, device="cuda")
        M.run_multi(Xd, Yd, 1.0, 0.0)
        Y = Yd.cpu().numpy()
        M.check_device()
    for j in range(7):
        check(A, X[j], Y[j])
