"""cbspmv_run_noalloc (the allocation-free product) against cbspmv_run, through the C ABI.

Some callers may not call cudaMalloc or any allocating routine when they run the product
(their device memory belongs to another allocator, or the path is latency-critical), so
the library offers one entry point whose scratch comes from a fixed array in the device
image. This file is collected last so that a failure here does not hide the other tests;
it must pass alone in a fresh process and after the rest of the suite."""
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


def cut_rows_matrix():
    # block rows far above one unit's budget, so the product needs the split-row scratch
    r, c = [], []
    for b, cols in ((0, 9000), (5, 30000)):
        rr = np.repeat(np.arange(16 * b, 16 * b + 16), cols // 16)
        r.append(rr); c.append((np.arange(rr.size) * 7919) % 40000)
    sp = I.random_csr(300, 40000, 0.001, 5)
    r.append(sp.rows()); c.append(sp.col)
    key = np.unique(np.concatenate(r) * 40000 + np.concatenate(c))
    return I.csr_from_coo(300, 40000, key // 40000, key % 40000, I.uniform_pm1(9, 2, key.size),
                          sum_duplicates=False)


@pytest.mark.parametrize("make", [cut_rows_matrix, lambda: I.laplacian2d(64), lambda: I.rmat(13, 16, seed=3)],
                         ids=["cut_rows", "laplace2d_64", "rmat13"])
def test_noalloc_matches_run_twice(env, make):
    bd, torch = env
    L = bd.lib()
    A = make()
    x = I.vector_x(A.n, 70)
    y0 = I.uniform_pm1(71, I.TAG_Y, A.m)
    with bd.BlockedMatrix(A) as M:
        st = M.stats()
        if make is cut_rows_matrix:
            assert st["n_split_rows"] >= 2
        xd = torch.from_numpy(x).cuda()
        yref = torch.from_numpy(y0.copy()).cuda()
        M.run(xd, yref, 1.25, -0.5)
        s = torch.cuda.current_stream().cuda_stream or None
        for call in range(2):                       # two calls in a row share the static scratch
            yd = torch.from_numpy(y0.copy()).cuda()
            status = L.cbspmv_run_noalloc(M.handle, xd.data_ptr(), yd.data_ptr(), 1.25, -0.5, s)
            assert status == 0, L.cbspmv_last_error().decode()
            torch.cuda.synchronize()
            M.check_device()
            got = yd.cpu().numpy()
            want = yref.cpu().numpy()
            _, scale = oracle.spmv(A, x)
            ok, worst = oracle.within_tolerance(got, want, scale, 1.25, -0.5, y0, RTOL)
            assert ok, f"call {call}: worst normalised error {worst:.3e}"


def test_noalloc_rejects_bad_arguments(env):
    bd, torch = env
    L = bd.lib()
    assert L.cbspmv_run_noalloc(None, None, None, 1.0, 0.0, None) == 1
    A = I.random_csr(40, 40, 0.2, 3)
    with bd.BlockedMatrix(A, device=-1) as H:
        assert L.cbspmv_run_noalloc(H.handle, None, None, 1.0, 0.0, None) == 1   # host-only handle
        assert b"device" in L.cbspmv_last_error()
    with bd.BlockedMatrix(A) as M:                  # x and y overlapping: rejected like cbspmv_run
        buf = torch.zeros(2 * A.n, dtype=torch.float64, device="cuda")
        assert L.cbspmv_run_noalloc(M.handle, buf.data_ptr(), buf.data_ptr() + 8 * 8, 1.0, 0.0, None) == 1
        assert b"overlap" in L.cbspmv_last_error()
        assert L.cbspmv_run_noalloc(M.handle, buf.data_ptr() + 4, buf.data_ptr() + 8 * A.n, 1.0, 0.0, None) == 1
