"""Randomised GPU parity: seeded random matrices (uniform, dense blocks on a sparse
background, power law), random analysis options, value types, alpha/beta and numbers of
right-hand sides, each product checked against the CPU oracle (FP64: 1e-12 of
sum |a x|; reduced types: the FP32 evaluation bound against the stored values)."""
import numpy as np
import pytest

import oracle
from oracle import lowprec as L
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def random_matrix(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 900)), int(rng.integers(1, 900))
    kind = seed % 3
    if kind == 0:
        return I.random_csr(m, n, float(rng.uniform(0.001, 0.4)), seed)
    if kind == 1:
        r, c = [], []
        for _ in range(int(rng.integers(1, 12))):
            r0, c0 = int(rng.integers(0, m)), int(rng.integers(0, n))
            h, w = int(rng.integers(1, 20)), int(rng.integers(1, 20))
            rr, cc = np.meshgrid(np.arange(r0, min(m, r0 + h)), np.arange(c0, min(n, c0 + w)), indexing="ij")
            r.append(rr.ravel()); c.append(cc.ravel())
        bg = I.random_csr(m, n, 0.01, seed + 1)
        r.append(bg.rows()); c.append(bg.col)
        r = np.concatenate(r); c = np.concatenate(c)
        key = np.unique(r.astype(np.int64) * n + c)
        return I.csr_from_coo(m, n, key // n, key % n, I.uniform_pm1(seed, 2, key.size), sum_duplicates=False)
    return I.rmat(int(rng.integers(6, 11)), 16, seed=seed)


@pytest.mark.parametrize("seed", range(24))
def test_random_products(env, seed):
    bd, torch = env
    rng = np.random.default_rng(5000 + seed)
    A = random_matrix(seed)
    th1 = int(rng.choice([0, 8, 32, 64]))
    th2 = max(th1, int(rng.choice([128, 200, 256])))
    opts = dict(col_agg=int(rng.choice([-1, 0, 1])), th1=th1, th2=th2,
                unit_work=int(rng.choice([0, 64, 300, 1024])), load_balance=bool(rng.integers(2)),
                record_layout=int(rng.choice([0, 1])))
    fmt = str(rng.choice(["f64", "f64", "f32", "bf16", "f16"]))
    alpha, beta = float(rng.choice([1.0, -0.75])), float(rng.choice([0.0, 0.5]))
    k = int(rng.integers(1, 6))
    vec = np.float64 if fmt == "f64" else np.float32
    X = np.stack([I.vector_x(A.n, 10 * seed + j) for j in range(k)]).astype(vec)
    Y0 = np.stack([I.uniform_pm1(20 * seed + j, I.TAG_Y, A.m) for j in range(k)]).astype(vec)
    with bd.BlockedMatrix(A, value_dtype=fmt, **opts) as M:
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.from_numpy(Y0.copy()).cuda()
        if k == 1:
            M.run(Xd[0], Yd[0], alpha, beta)
        else:
            M.run_multi(Xd, Yd, alpha, beta)
        Y = Yd.cpu().numpy()
        M.check_device()
    Ar = A if fmt == "f64" else L.stored_matrix(A, fmt)
    a_r = alpha if fmt == "f64" else float(np.float32(alpha))
    b_r = beta if fmt == "f64" else float(np.float32(beta))
    for j in range(k):
        x = X[j].astype(np.float64)
        y0 = Y0[j].astype(np.float64)
        yref, s = oracle.spmv(Ar, x, a_r, b_r, y0)
        if fmt == "f64":
            ok, worst = oracle.within_tolerance(Y[j], yref, s, alpha, beta, y0, 1e-12)
        else:
            scale = abs(a_r) * s + (np.abs(b_r * y0) if b_r != 0.0 else 0.0)
            ok, worst = L.within_bound(Y[j].astype(np.float64), yref, scale, L.fp32_bound(A))
        assert ok, f"seed {seed} ({fmt}, {opts}, k={k}): worst normalised error {worst:.3e}"
