"""GPU parity of the multi-vector, batched and device-input entry points against the CPU
oracle and against single-vector runs (same summation order, so bitwise equal)."""
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


def check(A, x, y, alpha=1.0, beta=0.0, y0=None):
    yref, s = oracle.spmv(A, x, alpha, beta, y0)
    ok, worst = oracle.within_tolerance(y, yref, s, alpha, beta, y0, RTOL)
    assert ok, f"worst normalised error {worst:.3e}"


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 8])
def test_run_multi_strided(env, k):
    bd, torch = env
    A = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    alpha, beta = 1.5, -0.5
    X = np.stack([I.vector_x(A.n, 40 + j) for j in range(k)])
    Y0 = np.stack([I.uniform_pm1(60 + j, I.TAG_Y, A.m) for j in range(k)])
    with bd.BlockedMatrix(A) as M:
        Xd = torch.zeros((k, A.n + 5), dtype=torch.float64, device="cuda")   # ldx = n + 5
        Yd = torch.zeros((k, A.m + 3), dtype=torch.float64, device="cuda")   # ldy = m + 3
        Xd[:, :A.n] = torch.from_numpy(X).cuda()
        Yd[:, :A.m] = torch.from_numpy(Y0).cuda()
        pad_before = Yd[:, A.m:].clone()
        M.run_multi(Xd[:, :A.n], Yd[:, :A.m], alpha, beta)
        Y = Yd[:, :A.m].cpu().numpy()
        assert torch.equal(Yd[:, A.m:], pad_before)         # nothing written past m
        for j in range(k):
            yj = torch.from_numpy(Y0[j].copy()).cuda()
            M.run(torch.from_numpy(X[j].copy()).cuda(), yj, alpha, beta)
            assert np.array_equal(Y[j], yj.cpu().numpy())
            check(A, X[j], Y[j], alpha, beta, Y0[j])
        M.check_device()


def test_run_multi_argument_checks(env):
    bd, torch = env
    A = I.laplacian2d(16)
    with bd.BlockedMatrix(A) as M:
        X = torch.zeros((2, A.n), dtype=torch.float64, device="cuda")
        Y = torch.zeros((2, A.m), dtype=torch.float64, device="cuda")
        lib = bd.lib()
        st = lib.cbspmv_run_multi(M.handle, 2, X.data_ptr(), A.n - 1, Y.data_ptr(), A.m, 1.0, 0.0, None)
        assert st == bd.CBSPMV_ERR_INVALID
        st = lib.cbspmv_run_multi(M.handle, 2, X.data_ptr(), A.n, X.data_ptr() + 8 * A.n, A.m, 1.0, 0.0, None)
        assert st == bd.CBSPMV_ERR_INVALID                  # Y overlaps X's second column
        assert lib.cbspmv_run_multi(M.handle, 0, None, A.n, None, A.m, 1.0, 0.0, None) == bd.CBSPMV_OK


def test_run_batched_matches_single_runs(env):
    bd, torch = env
    As = [I.laplacian3d(10), I.random_csr(333, 517, 0.2, 11), I.rmat(12, 16, seed=4)]
    ks = [1, 2, 3]
    alphas, betas = [1.0, -2.0, 0.5], [0.0, 1.0, -1.0]
    Ms = bd.analyze_batched(As)
    try:
        Xs, Ys, Y0s = [], [], []
        for i, (A, k) in enumerate(zip(As, ks)):
            X = np.stack([I.vector_x(A.n, 100 + 10 * i + j) for j in range(k)])
            Y0 = np.stack([I.uniform_pm1(200 + 10 * i + j, I.TAG_Y, A.m) for j in range(k)])
            Xs.append(torch.from_numpy(X if k > 1 else X[0]).cuda().contiguous())
            Ys.append(torch.from_numpy(Y0 if k > 1 else Y0[0]).cuda().contiguous())
            Y0s.append(Y0)
        bd.run_batched(Ms, Xs, Ys, alphas, betas)
        for i, (A, M, k) in enumerate(zip(As, Ms, ks)):
            Y = Ys[i].cpu().numpy().reshape(k, A.m)
            X = Xs[i].cpu().numpy().reshape(k, A.n)
            for j in range(k):
                yj = torch.from_numpy(Y0s[i][j].copy()).cuda()
                M.run(torch.from_numpy(X[j].copy()).cuda(), yj, alphas[i], betas[i])
                assert np.array_equal(Y[j], yj.cpu().numpy())
                check(A, X[j], Y[j], alphas[i], betas[i], Y0s[i][j])
            M.check_device()
    finally:
        for M in Ms:
            M.close()


def test_device_resident_csr_input(env):
    bd, torch = env
    A = I.rmat(12, 16, seed=8)
    Ad = I.CSR(A.m, A.n, torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
               torch.from_numpy(A.val).cuda())
    x = I.vector_x(A.n, 9)
    xd = torch.from_numpy(x).cuda()
    with bd.BlockedMatrix(Ad) as Md, bd.BlockedMatrix(A) as Mh:
        rp, col, val = Md.export_csr()
        assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
        assert np.array_equal(val.view(np.uint64), A.val.view(np.uint64))
        y1 = torch.zeros(A.m, dtype=torch.float64, device="cuda")
        y2 = torch.zeros(A.m, dtype=torch.float64, device="cuda")
        Md.run(xd, y1)
        Mh.run(xd, y2)
        assert torch.equal(y1, y2)
        check(A, x, y1.cpu().numpy())


@pytest.mark.parametrize("name", ["rmat12", "dense_70x45", "split_rows"])
def test_run_multi_structures(env, name):
    """4- and 2-vector passes on power-law rows, Dense tiles and split block rows."""
    bd, torch = env
    if name == "rmat12":
        A = I.rmat(12, 16, seed=4)
    elif name == "dense_70x45":
        A = I.random_csr(70, 45, 0.85, 6)
    else:
        r = np.repeat(np.arange(16), 900)
        c = np.tile(np.arange(900) * 3, 16)
        A = I.csr_from_coo(16, 2700, r, c, I.normal(5, I.TAG_VAL, r.size))
    k = 7
    X = np.stack([I.vector_x(A.n, 80 + j) for j in range(k)])
    Y0 = np.stack([I.uniform_pm1(90 + j, I.TAG_Y, A.m) for j in range(k)])
    with bd.BlockedMatrix(A, unit_work=256 if name == "split_rows" else 0) as M:
        if name == "split_rows":
            assert M.stats()["n_split_rows"] > 0
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.from_numpy(Y0.copy()).cuda()
        M.run_multi(Xd, Yd, 0.75, -1.25)
        Y = Yd.cpu().numpy()
        for j in range(k):
            yj = torch.from_numpy(Y0[j].copy()).cuda()
            M.run(torch.from_numpy(X[j].copy()).cuda(), yj, 0.75, -1.25)
            assert np.array_equal(Y[j], yj.cpu().numpy())
            check(A, X[j], Y[j], 0.75, -1.25, Y0[j])
        M.check_device()
