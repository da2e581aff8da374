"""Failure detection without a GPU fault: a bounded device wait that runs out of budget is
reported by cbspmv_check_device and leaves the device usable; a host-injected device
allocation failure makes cbspmv_analyze return CBSPMV_ERR_OOM and leak nothing."""
import os

import numpy as np
import pytest

import oracle
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu
ERR_OOM, ERR_TIMEOUT = 3, 5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def product(bd, torch, A, x, **opts):
    with bd.BlockedMatrix(A, **opts) as M:
        yd = torch.zeros(A.m, dtype=torch.float64 if x.dtype == np.float64 else torch.float32, device="cuda")
        M.run(torch.from_numpy(x).cuda(), yd)
        torch.cuda.synchronize()
        try:
            M.check_device()
            status = 0
        except bd.CbspmvError as e:
            status = e.status
        return yd.cpu().numpy(), status


def test_wait_budget_runs_out_and_device_stays_usable(env, monkeypatch):
    bd, torch = env
    A = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    x = I.vector_x(A.n, 5)
    # each warp's first wait is on a barrier nothing arrives at, with a budget of ~1 ms: it
    # gives up, the warp drains its own copies and stops
    monkeypatch.setenv("CBSPMV_WAIT_BUDGET_CYCLES", "2000000")
    monkeypatch.setenv("CBSPMV_TEST_STUCK_WAIT", "1")
    for dt in ("f64", "bf16"):
        _, status = product(bd, torch, A, x.astype(np.float64 if dt == "f64" else np.float32),
                            record_layout=True, value_dtype=dt)
        assert status == ERR_TIMEOUT
    monkeypatch.delenv("CBSPMV_WAIT_BUDGET_CYCLES")
    monkeypatch.delenv("CBSPMV_TEST_STUCK_WAIT")
    for rec in (True, False):             # the context is intact: full products are right again
        y, status = product(bd, torch, A, x, record_layout=rec)
        assert status == 0
        yref, s = oracle.spmv(A, x)
        assert oracle.within_tolerance(y, yref, s, rtol=1e-12)[0]


def test_forced_allocation_failure_leaks_nothing(env, monkeypatch):
    bd, torch = env
    A = I.rmat(12, 16, seed=6)
    x = I.vector_x(A.n, 7)
    product(bd, torch, A, x)              # warm: the context's own lazily loaded state
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n_fail in (0, 1, 2, 3, 5, 8):
        for rec in (False, True):
            monkeypatch.setenv("CBSPMV_FAIL_ALLOC_AFTER", str(n_fail))
            with pytest.raises(bd.CbspmvError) as ei:
                bd.BlockedMatrix(A, record_layout=rec)
            assert ei.value.status == ERR_OOM
    monkeypatch.delenv("CBSPMV_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 2 << 20
    # an injected failure past the call's last allocation changes nothing
    monkeypatch.setenv("CBSPMV_FAIL_ALLOC_AFTER", "1000")
    y, status = product(bd, torch, A, x)
    monkeypatch.delenv("CBSPMV_FAIL_ALLOC_AFTER")
    yref, s = oracle.spmv(A, x)
    assert status == 0 and oracle.within_tolerance(y, yref, s, rtol=1e-12)[0]
