"""GPU parity of the tensor-core multi-vector product (cbspmv_spmm, BF16 values, FP32 X
and Y, row-major) against the oracle.

Reference: the oracle's exact product of the stored BF16 values and the FP32 columns of X.
Bound per row, derived for this arithmetic: each x is split into three BF16 parts with
|x - (h + m + l)| <= 2^-25 |x| (a quarter of FP32's u); the MMA forms the 3 r products of
a row's r entries exactly and adds them, with the partial sums of up to 3 r / 16 + 3 r MMA
steps and the segment and alpha/beta merges, in FP32 whose adds may truncate (unit 2^-23):
gamma_{6 r + 16} with u = 2^-23 covers every add twice over. Checked also against the FP64
oracle on the FP64 values and x, where BF16's own rounding of the values is added."""
import numpy as np
import pytest

import oracle
from oracle import lowprec as L
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu
U23 = 2.0 ** -23


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def mma_bound(A):
    r = np.diff(np.asarray(A.row_ptr, dtype=np.int64)).astype(np.float64)
    k = 6 * r + 16
    return k * U23 / (1.0 - k * U23)


def heavy_block_rows():
    # block rows of 2,000 and 150 sub-blocks (cut into segments of 64) next to sparse rows
    r, c = [], []
    for b, cols in ((1, 32000), (4, 2400)):
        rr = np.repeat(np.arange(16 * b, 16 * b + 16), cols // 16)
        r.append(rr); c.append((np.arange(rr.size) * 7) % cols)
    sp = I.random_csr(100, 32000, 0.002, 17)
    r.append(sp.rows()); c.append(sp.col)
    key = np.unique(np.concatenate(r) * 32000 + np.concatenate(c))
    return I.csr_from_coo(100, 32000, key // 32000, key % 32000, I.uniform_pm1(18, 2, key.size),
                          sum_duplicates=False)


CASES = {
    "dense_70x45": lambda: I.random_csr(70, 45, 0.85, 6),
    "fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
    "rmat12": lambda: I.rmat(12, 16, seed=4),
    "laplace2d_64": lambda: I.laplacian2d(64),
    "heavy_block_rows": heavy_block_rows,
}


def check(A, X, Y, alpha, beta, Y0):
    """Every column of Y against the stored-value product and the FP64 oracle."""
    a32, b32 = float(np.float32(alpha)), float(np.float32(beta))
    Ar = L.stored_matrix(A, "bf16")
    bnd = mma_bound(A)
    worst = 0.0
    for j in range(X.shape[1]):
        x32 = X[:, j].astype(np.float64)
        y0 = Y0[:, j].astype(np.float64)
        y_ref, s = oracle.spmv(Ar, x32, a32, b32, y0)
        scale = abs(a32) * s + (np.abs(b32 * y0) if b32 != 0.0 else 0.0)
        ok, w = L.within_bound(Y[:, j], y_ref, scale, bnd)
        assert ok, f"column {j}: vs stored-value product, worst {w:.3e}"
        y64, s64 = oracle.spmv(A, x32, alpha, beta, y0)
        scale64 = abs(alpha) * s64 + (np.abs(beta * y0) if beta != 0.0 else 0.0)
        fac = L.UNIT_ROUNDOFF["bf16"] + 1.01 * bnd
        ok64, w64 = L.within_bound(Y[:, j], y64, scale64 * (1 + L.UNIT_ROUNDOFF["bf16"]), fac)
        assert ok64, f"column {j}: vs FP64 oracle, worst {w64:.3e}"
        worst = max(worst, w64)
    return worst


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("k", [1, 8, 32])
def test_spmm_against_oracle(env, name, k):
    bd, torch = env
    A = CASES[name]()
    X = np.stack([I.vector_x(A.n, 300 + j) for j in range(k)], axis=1).astype(np.float32)
    Y0 = np.stack([I.uniform_pm1(400 + j, I.TAG_Y, A.m) for j in range(k)], axis=1).astype(np.float32)
    for alpha, beta in ((1.0, 0.0), (-0.75, 0.5)):
        with bd.BlockedMatrix(A, value_dtype="bf16", plain_records=True) as M:
            Xd = torch.from_numpy(X).cuda()
            Yd = torch.from_numpy(Y0.copy()).cuda()
            M.spmm(Xd, Yd, alpha, beta)
            Y1 = Yd.cpu().numpy()
            Yd = torch.from_numpy(Y0.copy()).cuda()
            M.spmm(Xd, Yd, alpha, beta)
            M.check_device()
            assert np.array_equal(Yd.cpu().numpy(), Y1)       # deterministic
        check(A, X, Y1, alpha, beta, Y0)


def test_spmm_many_columns_and_leading_dimensions(env):
    """k = 40 (two launches of 32 and 8 columns) with padded leading dimensions; columns
    past k and padding are left untouched."""
    bd, torch = env
    A = I.fem_block_band(n_rows=3000, n_block_rows=1000, half_band=200, seed=5)
    k, ldx, ldy = 40, 44, 41
    Xf = np.zeros((A.n, ldx), np.float32)
    Xf[:, :k] = np.stack([I.vector_x(A.n, 500 + j) for j in range(k)], axis=1)
    Yf = np.full((A.m, ldy), 7.0, np.float32)
    with bd.BlockedMatrix(A, value_dtype="bf16", plain_records=True) as M:
        Xd = torch.from_numpy(Xf).cuda()
        Yd = torch.from_numpy(Yf.copy()).cuda()
        M.spmm(Xd[:, :k], Yd[:, :k])
        Y = Yd.cpu().numpy()
    assert np.all(Y[:, k:] == 7.0)
    check(A, Xf[:, :k], Y[:, :k], 1.0, 0.0, np.zeros((A.m, k), np.float32))


def test_spmm_rejects_other_handles(env):
    bd, torch = env
    A = I.random_csr(50, 40, 0.2, 3)
    X = torch.zeros((40, 8), dtype=torch.float32, device="cuda")
    Y = torch.zeros((50, 8), dtype=torch.float32, device="cuda")
    with bd.BlockedMatrix(A, value_dtype="f32", plain_records=True) as M:
        with pytest.raises(bd.CbspmvError) as ei:
            M.spmm(X, Y)
        assert ei.value.status == 6
    R = I.fem_block_band(n_rows=600, n_block_rows=200, half_band=50, seed=3)
    with bd.BlockedMatrix(R, value_dtype="bf16", record_layout=1) as M:   # records with direct units
        if M.stats()["n_direct_units"]:
            with pytest.raises(bd.CbspmvError) as ei:
                M.spmm(torch.zeros((R.n, 8), dtype=torch.float32, device="cuda"),
                       torch.zeros((R.m, 8), dtype=torch.float32, device="cuda"))
            assert ei.value.status == 6
    with bd.BlockedMatrix(A, value_dtype="bf16") as M:   # lane streams (the default)
        with pytest.raises(bd.CbspmvError) as ei:
            M.spmm(X, Y)
        assert ei.value.status == 6
    with bd.BlockedMatrix(A, value_dtype="bf16", plain_records=True) as M:
        buf = torch.zeros((60, 8), dtype=torch.float32, device="cuda")
        with pytest.raises(bd.CbspmvError):
            M.spmm(buf[:40], buf[5:55])            # X and Y overlap
