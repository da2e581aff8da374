"""Device-side analysis (cbspmv_analyze of a CSR in device memory, lane-stream layout):
the GPU builds the block-row merge, tiling, aggregation and the lane programs; the host
keeps the units and the load balance.

Every case is compared three ways: the blocked structure against oracle/blocked.py
(Sec. 3.3: aggregation decision, tiles, formats, restore_cols), the CSR exported back from
the handle bit for bit against the input, and the handle against the host-analysed handle
of the same matrix (same statistics, bit-identical products, since both build the same
lane arrays), with the product also checked against the FP64 oracle.
"""
import types

import numpy as np
import pytest

import oracle
from oracle import blocked as B
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu
ERR_NOT_CANONICAL = 2
ERR_OOM = 3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def on_device(torch, A):
    return types.SimpleNamespace(m=A.m, n=A.n, row_ptr=torch.from_numpy(np.asarray(A.row_ptr, np.int64)).cuda(),
                                 col=torch.from_numpy(np.asarray(A.col, np.int32)).cuda(),
                                 val=torch.from_numpy(np.asarray(A.val, np.float64)).cuda())


def product(torch, M, x):
    y = torch.zeros(M.m, dtype=torch.float64, device="cuda")
    M.run(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    M.check_device()
    return y.cpu().numpy()


def compare(env, A, **opts):
    bd, torch = env
    x = I.vector_x(A.n, 31)
    with bd.BlockedMatrix(on_device(torch, A), **opts) as Md, bd.BlockedMatrix(A, **opts) as Mh:
        sd, sh = Md.stats(), Mh.stats()
        assert sd["analyzed_on_device"] == 1 and sh["analyzed_on_device"] == 0
        for k in sh:
            if k not in ("analyze_ms", "analyzed_on_device"):
                assert sd[k] == sh[k], k
        # blocked structure of the device-analysed handle against the oracle
        S = B.blocked_structure(A, th0=opts.get("th0", 0.15), th1=opts.get("th1", 32), th2=opts.get("th2", 128),
                                col_agg=opts.get("col_agg", -1))
        got = Md.export_blocked()
        assert got["aggregated"] == S.aggregated
        assert np.array_equal(got["blk_row"], S.tile_brow)
        assert np.array_equal(got["blk_col"], S.tile_bcol)
        assert np.array_equal(got["nnz"], S.tile_nnz)
        assert np.array_equal(got["type"], S.tile_fmt)
        if S.aggregated:
            assert np.array_equal(got["cols_offset"], S.cols_offset)
            assert np.array_equal(got["restore_cols"], S.restore_cols)
        assert sd["super_sparse_fraction"] == pytest.approx(B.super_sparse_fraction(A, opts.get("th1", 32)), abs=0)
        # CSR round trip, bit for bit
        rp, col, val = Md.export_csr()
        assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
        assert np.array_equal(val.view(np.uint64), np.asarray(A.val, np.float64).view(np.uint64))
        if A.m == 0:
            return sd
        yd, yh = product(torch, Md, x), product(torch, Mh, x)
    assert np.array_equal(yd.view(np.uint64), yh.view(np.uint64))
    yref, s = oracle.spmv(A, x)
    assert oracle.within_tolerance(yd, yref, s, rtol=1e-12)[0]
    return sd


def dense_rows(m, n, rows, seed):
    """Rows listed in `rows` hold every column; the others a few entries."""
    rng = np.random.default_rng(seed)
    rp, cols = [0], []
    for r in range(m):
        c = np.arange(n) if r in rows else np.sort(rng.choice(n, size=min(n, 3), replace=False))
        cols.append(c)
        rp.append(rp[-1] + c.size)
    col = np.concatenate(cols).astype(np.int32)
    return I.CSR(m, n, np.array(rp, np.int64), col, rng.uniform(-1, 1, col.size))


CASES = {
    "laplace2d_64": lambda: I.laplacian2d(64),
    "ragged_203x157": lambda: I.random_csr(203, 157, 0.07, 5),
    "dense_70x45": lambda: I.random_csr(70, 45, 0.85, 6),
    "mixed_333x517": lambda: I.random_csr(333, 517, 0.2, 11),
    "rmat12": lambda: I.rmat(12, 16, seed=4),
    "rmat14_large_block_rows": lambda: I.rmat(14, 16, seed=9),
    "fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
    "one_row_5000": lambda: I.random_csr(1, 5000, 0.9, 7),
    "one_col": lambda: I.random_csr(3000, 1, 0.5, 8),
    "long_rows_one_block_row": lambda: dense_rows(40, 3000, {0, 3, 17, 31, 39}, 13),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("col_agg", [-1, 0, 1])
def test_device_analysis_matches_host_and_oracle(env, name, col_agg):
    compare(env, CASES[name](), col_agg=col_agg)


@pytest.mark.parametrize("unit_work", [64, 512, 4096, 16384])
def test_device_analysis_unit_sizes(env, unit_work):
    """Small units cut block rows into many parts (split rows, column ranges of a row)."""
    compare(env, dense_rows(64, 2000, {1, 2, 20, 47}, 21), unit_work=unit_work)
    compare(env, I.rmat(12, 16, seed=5), unit_work=unit_work, col_agg=1)


@pytest.mark.parametrize("th1,th2", [(0, 0), (256, 256), (8, 40)])
def test_device_analysis_thresholds(env, th1, th2):
    compare(env, I.random_csr(300, 280, 0.3, 44), th1=th1, th2=th2)


def test_device_analysis_degenerate(env):
    compare(env, I.CSR(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)))
    compare(env, I.CSR(37, 50, np.zeros(38, np.int64), np.zeros(0, np.int32), np.zeros(0)))
    compare(env, I.random_csr(17, 1, 1.0, 3))
    compare(env, I.CSR(1, 1, np.array([0, 1], np.int64), np.zeros(1, np.int32), np.array([2.5])))


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", ["mixed_333x517", "rmat14_large_block_rows", "fem_small"])
def test_device_analysis_reduced_types(env, fmt, name):
    """record_layout 2 with FP32 / BF16 / FP16 values: the device analysis rounds every value
    like the host analysis (same bits), so both handles give bit-identical products."""
    bd, torch = env
    from oracle import lowprec as L
    A = CASES[name]()
    x = I.vector_x(A.n, 5).astype(np.float32)
    with bd.BlockedMatrix(on_device(torch, A), value_dtype=fmt, record_layout=2) as Md, \
            bd.BlockedMatrix(A, value_dtype=fmt, record_layout=2) as Mh:
        sd, sh = Md.stats(), Mh.stats()
        assert sd["analyzed_on_device"] == 1
        for k in sh:
            if k not in ("analyze_ms", "analyzed_on_device"):
                assert sd[k] == sh[k], k
        rp, col, val = Md.export_csr()
        assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
        assert np.array_equal(val, L.round_to_format(A.val, fmt))
        ys = []
        for M in (Md, Mh):
            y = torch.zeros(A.m, dtype=torch.float32, device="cuda")
            M.run(torch.from_numpy(x).cuda(), y)
            torch.cuda.synchronize()
            M.check_device()
            ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0].view(np.uint32), ys[1].view(np.uint32))


def test_device_analysis_value_map(env):
    """keep_value_map on the device: new values through cbspmv_update_values give the same
    bits as a host-analysed handle given the same values."""
    bd, torch = env
    A = I.rmat(13, 16, seed=6)
    x = I.vector_x(A.n, 3)
    v2 = I.uniform_pm1(77, I.TAG_VAL, A.nnz)
    with bd.BlockedMatrix(on_device(torch, A), keep_value_map=True) as Md, \
            bd.BlockedMatrix(A, keep_value_map=True) as Mh:
        for M in (Md, Mh):
            M.update_values(torch.from_numpy(v2).cuda())
        yd, yh = product(torch, Md, x), product(torch, Mh, x)
    assert np.array_equal(yd.view(np.uint64), yh.view(np.uint64))
    A2 = I.CSR(A.m, A.n, A.row_ptr, A.col, v2)
    yref, s = oracle.spmv(A2, x)
    assert oracle.within_tolerance(yd, yref, s, rtol=1e-12)[0]


def bad(A, **kw):
    d = dict(m=A.m, n=A.n, row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val.copy())
    d.update(kw)
    return types.SimpleNamespace(**d)


def test_device_analysis_rejects_non_canonical(env):
    """Invalid CSR arrays are found on the device before any other use of them (every read
    stays inside the arrays) and the device stays usable."""
    bd, torch = env
    A = I.random_csr(100, 90, 0.1, 2)
    r = int(np.argmax(np.diff(A.row_ptr) >= 2))
    k = int(A.row_ptr[r])
    unsorted = A.col.copy(); unsorted[k], unsorted[k + 1] = unsorted[k + 1], unsorted[k]
    dup = A.col.copy(); dup[k + 1] = dup[k]
    big = A.col.copy(); big[k] = A.n
    neg = A.col.copy(); neg[k] = -1
    dec = A.row_ptr.copy(); dec[r + 1] = dec[r] - 1 if dec[r] > 0 else dec[r]; dec[5] = dec[6] + 1
    end = A.row_ptr.copy(); end[-1] -= 1
    for C in (bad(A, col=unsorted), bad(A, col=dup), bad(A, col=big), bad(A, col=neg), bad(A, row_ptr=dec),
              bad(A, row_ptr=end)):
        with pytest.raises(bd.CbspmvError) as ei:
            bd.BlockedMatrix(on_device(torch, C))
        assert ei.value.status == ERR_NOT_CANONICAL
    compare(env, A)


def test_device_analysis_allocation_failure_leaks_nothing(env, monkeypatch):
    bd, torch = env
    A = I.rmat(14, 16, seed=9)   # has block rows merged in global memory
    Ad = on_device(torch, A)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n_fail in range(0, 60):
        monkeypatch.setenv("CBSPMV_FAIL_ALLOC_AFTER", str(n_fail))
        try:
            M = bd.BlockedMatrix(Ad)
        except bd.CbspmvError as e:
            assert e.status == ERR_OOM
        else:
            M.close()
            break
    else:
        raise AssertionError("the analysis allocates more than 60 buffers")
    monkeypatch.delenv("CBSPMV_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 2 << 20
    compare(env, A)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["fem3x3_band_1m", "rmat_s21"])
def test_device_analysis_full_size(env, name):
    """The full-size configurations: same statistics and bit-identical products as the
    host analysis, CSR round trip bit for bit."""
    bd, torch = env
    A, x = I.config_matrix(name)
    with bd.BlockedMatrix(on_device(torch, A)) as Md:
        sd = Md.stats()
        rp, col, val = Md.export_csr()
        assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
        assert np.array_equal(val.view(np.uint64), A.val.view(np.uint64))
        del rp, col, val
        yd = product(torch, Md, x)
    with bd.BlockedMatrix(A) as Mh:
        sh = Mh.stats()
        yh = product(torch, Mh, x)
    for k in sh:
        if k not in ("analyze_ms", "analyzed_on_device"):
            assert sd[k] == sh[k], k
    assert np.array_equal(yd.view(np.uint64), yh.view(np.uint64))
    assert sd["analyze_ms"] < sh["analyze_ms"]
