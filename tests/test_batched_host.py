"""CPU tests of the batched and multi-vector entry points that need no GPU: batched analysis
into host-only handles (same structure as one-at-a-time analysis, clean failure) and the
argument checks of the run calls."""
import numpy as np
import pytest

from paper_2605_18515_gb300 import build, inputs as I


@pytest.fixture(scope="module")
def bd():
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding


def mats():
    return [I.laplacian2d(20), I.random_csr(203, 157, 0.07, 5), I.rmat(10, 16, seed=4)]


def test_analyze_batched_equals_single(bd):
    As = mats()
    Ms = bd.analyze_batched(As, device=-1)
    try:
        for A, M in zip(As, Ms):
            with bd.BlockedMatrix(A, device=-1) as S:
                a, b = M.export_blocked(), S.export_blocked()
                for key in ("blk_row", "blk_col", "nnz", "type", "cols_offset", "restore_cols"):
                    assert np.array_equal(a[key], b[key])
                assert M.stats()["n_units"] == S.stats()["n_units"]
            rp, col, val = M.export_csr()
            assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
            assert np.array_equal(val.view(np.uint64), A.val.view(np.uint64))
    finally:
        for M in Ms:
            M.close()


def test_analyze_batched_failure_names_matrix(bd):
    As = mats()
    bad = I.CSR(3, 3, np.array([0, 2, 2, 2]), np.array([1, 0], np.int32), np.array([1.0, 2.0]))
    As.insert(1, bad)                        # unsorted columns in row 0
    with pytest.raises(bd.CbspmvError) as e:
        bd.analyze_batched(As, device=-1)
    assert e.value.status == bd.CBSPMV_ERR_NOT_CANONICAL
    assert "matrix 1" in str(e.value)


def test_analyze_batched_empty(bd):
    assert bd.analyze_batched([], device=-1) == []


def test_run_calls_reject_host_only_handles(bd):
    import ctypes
    A = I.laplacian2d(8)
    with bd.BlockedMatrix(A, device=-1) as M:
        lib = bd.lib()
        st = lib.cbspmv_run_multi(M.handle, 1, 16, A.n, 4096, A.m, 1.0, 0.0, None)
        assert st == bd.CBSPMV_ERR_INVALID
        st = lib.cbspmv_run_multi(M.handle, -1, 16, A.n, 4096, A.m, 1.0, 0.0, None)
        assert st == bd.CBSPMV_ERR_INVALID
        hs = (ctypes.c_void_p * 1)(M.handle)
        xs = (ctypes.c_void_p * 1)(16)
        ys = (ctypes.c_void_p * 1)(4096)
        al = (ctypes.c_double * 1)(1.0)
        be = (ctypes.c_double * 1)(0.0)
        st = lib.cbspmv_run_batched(1, ctypes.addressof(hs), None, ctypes.addressof(xs),
                                    ctypes.addressof(ys), ctypes.addressof(al), ctypes.addressof(be), None)
        assert st == bd.CBSPMV_ERR_INVALID
        assert "problem 0" in lib.cbspmv_last_error().decode()
        assert lib.cbspmv_run_batched(0, None, None, None, None, None, None, None) == bd.CBSPMV_OK


def test_server_options_are_checked_without_a_device(bd):
    import ctypes
    o = bd.ServerOpts()
    assert bd.lib().cbspmv_server_default_opts(ctypes.byref(o)) == bd.CBSPMV_OK
    assert o.max_inflight == 64 and o.cg_inner_dtype == 2 and o.max_outer == 30
    s = ctypes.c_void_p(None)
    for field, bad in (("max_inflight", 0), ("max_inflight", 65), ("inner_tol", 0.0), ("max_outer", 0),
                       ("memory_budget", 1024)):
        o2 = bd.ServerOpts()
        bd.lib().cbspmv_server_default_opts(ctypes.byref(o2))
        setattr(o2, field, bad)
        assert bd.lib().cbspmv_server_create(ctypes.byref(o2), ctypes.byref(s)) == bd.CBSPMV_ERR_INVALID
        assert s.value is None
    o.device = 9999                      # no such device: an error status, never a crash
    assert bd.lib().cbspmv_server_create(ctypes.byref(o), ctypes.byref(s)) in (bd.CBSPMV_ERR_INVALID,
                                                                               bd.CBSPMV_ERR_CUDA)
    assert s.value is None
    assert bd.lib().cbspmv_server_destroy(None) == bd.CBSPMV_OK
