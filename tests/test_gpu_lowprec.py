"""GPU parity of the reduced-precision value types (FP32 / BF16 / FP16 storage, FP32 x, y
and accumulation) against the oracle.

Two checks per result: (1) against the exact product of the stored values and the FP32 x
(the oracle's FP64 CSR product of the rounded matrix) within the FP32 evaluation bound
gamma_{k+10} per row; (2) against the FP64 oracle on the original FP64 values and x
within u_storage + u_fp32 + that bound, the error of the storage format itself."""
import numpy as np
import pytest

import oracle
from oracle import lowprec as L
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu
FMTS = ["f32", "bf16", "f16"]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32)


def check_lowprec(A, fmt, x, y_gpu, alpha=1.0, beta=0.0, y0=None, rows=None):
    """Both acceptance checks for the rows `rows` (all rows when None)."""
    a32, b32 = float(np.float32(alpha)), float(np.float32(beta))
    x32 = f32(x).astype(np.float64)
    y032 = None if y0 is None else f32(y0).astype(np.float64)
    Ar = L.stored_matrix(A, fmt)
    if rows is None:
        y_ref, s = oracle.spmv(Ar, x32, a32, b32, y032)
        y64, s64 = oracle.spmv(A, np.asarray(x, np.float64), alpha, beta, y0)
        bnd = L.fp32_bound(A)
        yg = np.asarray(y_gpu, np.float64)
        y0r = y032
        y0o = y0
    else:
        y_ref, s = oracle.spmv_rows(Ar, x32, rows, a32, b32, y032)
        y64, s64 = oracle.spmv_rows(A, np.asarray(x, np.float64), rows, alpha, beta, y0)
        bnd = L.fp32_bound(A)[rows]
        yg = np.asarray(y_gpu, np.float64)[rows]
        y0r = None if y032 is None else y032[rows]
        y0o = None if y0 is None else np.asarray(y0)[rows]
    scale = abs(a32) * s + (np.abs(b32 * y0r) if b32 != 0.0 else 0.0)
    ok, worst = L.within_bound(yg, y_ref, scale, bnd)
    assert ok, f"{fmt}: vs stored-value product, worst normalised error {worst:.3e}"
    scale64 = abs(alpha) * s64 + (np.abs(beta * y0o) if beta != 0.0 else 0.0)
    fac = L.UNIT_ROUNDOFF[fmt] + L.U32 + 1.01 * bnd + 4 * L.U32 * L.UNIT_ROUNDOFF[fmt]
    ok64, worst64 = L.within_bound(yg, y64, scale64 * (1 + L.UNIT_ROUNDOFF[fmt]), fac)
    assert ok64, f"{fmt}: vs FP64 oracle, worst normalised error {worst64:.3e}"
    return worst64


def run_lp(env, A, fmt, x, alpha=1.0, beta=0.0, y0=None, **opts):
    bd, torch = env
    with bd.BlockedMatrix(A, value_dtype=fmt, **opts) as M:
        xd = torch.from_numpy(f32(x)).cuda()
        yd = torch.from_numpy(f32(y0) if y0 is not None else np.zeros(A.m, np.float32)).cuda()
        M.run(xd, yd, alpha, beta)
        y = yd.cpu().numpy()
        M.check_device()
    return y


CASES = {
    "laplace2d_64": lambda: I.laplacian2d(64),
    "ragged_203x157": lambda: I.random_csr(203, 157, 0.07, 5),
    "dense_70x45": lambda: I.random_csr(70, 45, 0.85, 6),
    "mixed_333x517": lambda: I.random_csr(333, 517, 0.2, 11),
    "rmat12": lambda: I.rmat(12, 16, seed=4),
    "fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
}


LAYOUTS = {"records": 1, "lanes": 0}


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_lowprec_parity(env, fmt, name, layout):
    A = CASES[name]()
    x = I.vector_x(A.n, 31)
    y = run_lp(env, A, fmt, x, record_layout=LAYOUTS[layout])
    check_lowprec(A, fmt, x, y)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("col_agg", [0, 1])
@pytest.mark.parametrize("alpha,beta", [(2.5, 0.0), (-0.5, 0.25), (0.0, 2.0)])
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_lowprec_alpha_beta_aggregation(env, fmt, col_agg, alpha, beta, layout):
    A = I.random_csr(333, 517, 0.05, 13)
    x = I.vector_x(A.n, 32)
    y0 = I.uniform_pm1(33, I.TAG_Y, A.m)
    y = run_lp(env, A, fmt, x, alpha, beta, y0, col_agg=col_agg, record_layout=LAYOUTS[layout])
    check_lowprec(A, fmt, x, y, alpha, beta, y0)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_lowprec_split_rows_deterministic(env, fmt, layout):
    bd, torch = env
    r = np.repeat(np.arange(16), 900)
    c = np.tile(np.arange(900) * 3, 16)
    A = I.csr_from_coo(16, 2700, r, c, I.normal(5, I.TAG_VAL, r.size))
    x = I.vector_x(A.n, 34)
    with bd.BlockedMatrix(A, value_dtype=fmt, unit_work=256, record_layout=LAYOUTS[layout]) as M:
        assert M.stats()["n_split_rows"] > 0
        xd = torch.from_numpy(f32(x)).cuda()
        outs = []
        for _ in range(3):
            yd = torch.zeros(A.m, dtype=torch.float32, device="cuda")
            M.run(xd, yd)
            outs.append(yd.cpu().numpy())
        M.check_device()
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    check_lowprec(A, fmt, x, outs[0])


@pytest.mark.parametrize("fmt,k", [("bf16", 3), ("f32", 4), ("f16", 7)])
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_lowprec_run_multi_and_host(env, fmt, k, layout):
    bd, torch = env
    A = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    X = np.stack([f32(I.vector_x(A.n, 50 + j)) for j in range(k)])
    with bd.BlockedMatrix(A, value_dtype=fmt, record_layout=LAYOUTS[layout]) as M:
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros((k, A.m), dtype=torch.float32, device="cuda")
        M.run_multi(Xd, Yd, 1.0, 0.0)
        Y = Yd.cpu().numpy()
        for j in range(k):
            yh = M.run_host(X[j], np.zeros(A.m, np.float32))
            assert np.array_equal(yh, Y[j])
            check_lowprec(A, fmt, X[j], Y[j])


@pytest.mark.slow
def test_lowprec_full_size_fem(env):
    bd, torch = env
    A, x = I.config_matrix("fem3x3_band_1m")
    deg = np.diff(A.row_ptr)
    rows = np.unique(np.concatenate([np.arange(64), np.arange(A.m - 64, A.m),
                                     (I.uniform01(6, 9, 20000) * A.m).astype(np.int64), np.argsort(deg)[-200:]]))
    for fmt, layout in [(f, l) for f in FMTS for l in LAYOUTS.values()]:
        with bd.BlockedMatrix(A, value_dtype=fmt, record_layout=layout) as M:
            xd = torch.from_numpy(f32(x)).cuda()
            yd = torch.empty(A.m, dtype=torch.float32, device="cuda")
            M.run(xd, yd)
            y = yd.cpu().numpy()
            M.check_device()
        check_lowprec(A, fmt, x, y, rows=rows)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("steps", [1, 3, 4, 5, 7, 8, 9, 12, 15, 16, 17, 23])
@pytest.mark.parametrize("short", [0, 5])
def test_lane_layout_every_tail_length(env, fmt, steps, short):
    """Lane-stream units of every length modulo the 8-step group: one block row of 16 rows
    with 32 * steps - short entries (short > 0: some lanes' runs one step shorter), so the
    unit's last steps % 8 steps take the compact tail of the layout (no padding to a group),
    and a unit shorter than a group is nothing but a tail."""
    W = 32 * steps - short
    per = np.full(16, W // 16)
    per[: W % 16] += 1
    r = np.repeat(np.arange(16), per)
    c = np.concatenate([np.linspace(0, 511, k).astype(np.int64) for k in per])   # distinct per row
    A = I.csr_from_coo(16, 4000, r, c, I.normal(40 + steps, I.TAG_VAL, r.size))
    assert A.nnz == W
    x = I.vector_x(A.n, 35)
    for agg in (0, 1):
        bd, _ = env
        with bd.BlockedMatrix(A, value_dtype=fmt, record_layout=2, col_agg=agg) as M:
            st = M.stats()
            assert st["lane_layout"] == 1 and st["n_units"] == 1 and st["fma_slots"] == 32 * steps
        y = run_lp(env, A, fmt, x, record_layout=2, col_agg=agg)
        check_lowprec(A, fmt, x, y)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("name", ["rmat12", "split_rows", "plain_333x517"])
def test_lane_layout_four_vector_passes(env, fmt, name):
    """Lane-stream handles of the reduced types take their columns in passes of four (then
    single columns), in cbspmv_run_multi and cbspmv_run_batched: every column equals its
    single-vector run bit for bit (same summation order) and meets the oracle's bound. Cases:
    power-law rows with 32-bit gather lists, block rows cut into parts (combine of four
    columns), plain sub-blocks without aggregation, with alpha and beta."""
    bd, torch = env
    if name == "rmat12":
        A, kw = I.rmat(12, 16, seed=4), {}
    elif name == "split_rows":
        r = np.repeat(np.arange(16), 900)
        c = np.tile(np.arange(900) * 3, 16)
        A, kw = I.csr_from_coo(16, 2700, r, c, I.normal(5, I.TAG_VAL, r.size)), {"unit_work": 256}
    else:
        A, kw = I.random_csr(333, 517, 0.2, 11), {"col_agg": 0}
    k, alpha, beta = 6, 0.75, -1.25
    X = np.stack([f32(I.vector_x(A.n, 80 + j)) for j in range(k)])
    Y0 = np.stack([f32(I.uniform_pm1(90 + j, I.TAG_Y, A.m)) for j in range(k)])
    with bd.BlockedMatrix(A, value_dtype=fmt, record_layout=2, **kw) as M:
        assert M.stats()["lane_layout"] == 1
        if name == "split_rows":
            assert M.stats()["n_split_rows"] > 0
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.from_numpy(Y0.copy()).cuda()
        M.run_multi(Xd, Yd, alpha, beta)
        Y = Yd.cpu().numpy()
        Yb = torch.from_numpy(Y0.copy()).cuda()
        bd.run_batched([M], [Xd], [Yb], [alpha], [beta])
        assert np.array_equal(Yb.cpu().numpy(), Y)
        for j in range(k):
            yj = torch.from_numpy(Y0[j].copy()).cuda()
            M.run(torch.from_numpy(X[j].copy()).cuda(), yj, alpha, beta)
            assert np.array_equal(Y[j], yj.cpu().numpy())
            check_lowprec(A, fmt, X[j], Y[j], alpha, beta, Y0[j])
        M.check_device()
