"""GPU tests of the serving engine: y = Ax requests equal the library's own product bit
for bit, CG solves reach ||b - A x|| <= 1e-8 ||b|| measured by the FP64 CPU oracle, every
result is the same alone and in a mix of concurrent requests, and admission respects the
memory budget."""
import numpy as np
import pytest

import oracle
from paper_2605_18515_gb300 import build, inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding, torch


def true_rel_residual(A, x, b):
    y, _ = oracle.spmv(A, x)
    return float(np.linalg.norm(b - y) / np.linalg.norm(b))


def solo_product(bd, torch, A, x, alpha=1.0, beta=0.0, y0=None):
    with bd.BlockedMatrix(A) as M:
        yd = torch.from_numpy(np.array(y0 if y0 is not None else np.zeros(A.m))).cuda()
        M.run(torch.from_numpy(x).cuda(), yd, alpha, beta)
        return yd.cpu().numpy()


def test_mixed_requests(env):
    bd, torch = env
    L1, L2 = I.laplacian3d(12), I.laplacian3d(16)
    R = I.random_csr(700, 500, 0.02, 3)
    F = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    with bd.Server(max_inflight=64) as S:
        ids = [S.register(A) for A in (L1, L2, R, F)]
        reqs = []
        for i in range(24):
            if i % 3 == 0:
                A, mid = (L1, ids[0]) if i % 2 else (L2, ids[1])
                b = I.uniform_pm1(100 + i, I.TAG_RHS, A.n)
                t, x = S.submit_cg(mid, b, TOL)
                reqs.append(("cg", A, t, b, x))
            else:
                A, mid = [(L1, ids[0]), (R, ids[2]), (F, ids[3])][i % 3 - 1 + (i % 2)]
                x = I.vector_x(A.n, 200 + i)
                y0 = I.uniform_pm1(300 + i, I.TAG_Y, A.m)
                alpha, beta = (1.0, 0.0) if i % 4 else (-0.5, 2.0)
                t, y = S.submit_spmv(mid, x, y0.copy(), alpha, beta)
                reqs.append(("spmv", A, t, (x, y0, alpha, beta), y))
        for kind, A, t, inp, out in reqs:
            r = S.wait(t, 120000)
            assert r["done"] and r["status"] == 0, r
            if kind == "cg":
                assert true_rel_residual(A, out, inp) <= TOL * 1.0001
                assert r["rel_residual"] <= TOL
            else:
                x, y0, alpha, beta = inp
                assert np.array_equal(out, solo_product(bd, torch, A, x, alpha, beta, y0))
                yref, s = oracle.spmv(A, x, alpha, beta, y0)
                assert oracle.within_tolerance(out, yref, s, alpha, beta, y0, 1e-12)[0]
        st = S.stats()
        assert st["completed"] == len(reqs) and st["max_inflight_seen"] > 1


def test_result_same_alone_and_in_mix(env):
    bd, torch = env
    L = I.laplacian3d(14)
    b = I.uniform_pm1(7, I.TAG_RHS, L.n)
    with bd.Server() as S:
        mid = S.register(L)
        t, x_alone = S.submit_cg(mid, b, TOL)
        r_alone = S.wait(t)
        others = [S.submit_cg(mid, I.uniform_pm1(50 + i, I.TAG_RHS, L.n), TOL) for i in range(6)]
        t2, x_mix = S.submit_cg(mid, b, TOL)
        others += [S.submit_cg(mid, I.uniform_pm1(70 + i, I.TAG_RHS, L.n), TOL) for i in range(6)]
        r_mix = S.wait(t2)
        for t_o, _ in others:
            assert S.wait(t_o)["status"] == 0
    assert r_alone["status"] == 0 and r_mix["status"] == 0
    assert r_alone["iterations"] == r_mix["iterations"]
    assert np.array_equal(x_alone, x_mix)
    assert true_rel_residual(L, x_mix, b) <= TOL * 1.0001


def test_mixed_precision_cg_needs_few_refinements(env):
    bd, _ = env
    L = I.laplacian3d(20)
    b = I.uniform_pm1(9, I.TAG_RHS, L.n)
    with bd.Server(cg_inner_dtype="bf16", inner_tol=1e-4) as S:
        t, x = S.submit_cg(S.register(L), b, TOL)
        r = S.wait(t)
    assert r["status"] == 0 and 1 <= r["refinements"] <= 6
    assert true_rel_residual(L, x, b) <= TOL * 1.0001


def cg_iterations_fp64(A, b, rel):
    """Iterations of textbook CG in FP64 from x = 0 until its residual is rel ||b||."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    r = b.copy()
    p = r.copy()
    rr = rr0 = float(r @ r)
    k = 0
    while rr > rel * rel * rr0:
        q = M @ p
        al = rr / float(p @ q)
        r -= al * q
        t = float(r @ r)
        p = r + (t / rr) * p
        rr = t
        k += 1
    return k


def test_later_corrections_stop_at_the_gap_to_tol(env):
    """A correction after the first only has to close the gap between its starting residual
    and tol ||b|| (with 0.3 to spare): with inner_tol 1e-6 and tol 1e-8 the first correction
    takes the iterations of a 1e-6 solve (N) and the second those of a ~3e-3 one, so the
    solve takes two refinements and well under the 2N iterations of two full-depth
    corrections (an FP32 simulation of a 20^3 Laplacian with another uniform right-hand side:
    84 iterations against 128, N = 63)."""
    bd, _ = env
    L = I.laplacian3d(20)
    b = I.uniform_pm1(9, I.TAG_RHS, L.n)
    with bd.Server(cg_inner_dtype="bf16", inner_tol=1e-6) as S:
        t, x = S.submit_cg(S.register(L), b, TOL)
        r = S.wait(t)
    n1 = cg_iterations_fp64(L, b, 1e-6)
    assert r["status"] == 0 and r["refinements"] == 2, r
    assert r["iterations"] <= 1.5 * n1, (r["iterations"], n1)
    assert true_rel_residual(L, x, b) <= TOL * 1.0001


def test_fp64_one_at_a_time_mode(env):
    bd, _ = env
    L = I.laplacian3d(12)
    b = I.uniform_pm1(11, I.TAG_RHS, L.n)
    with bd.Server(max_inflight=1, cg_inner_dtype="f64", inner_tol=1e-9) as S:
        mid = S.register(L)
        ts = [S.submit_cg(mid, b, TOL) for _ in range(3)]
        rs = [S.wait(t) for t, _ in ts]
        assert S.stats()["max_inflight_seen"] == 1
    for (t, x), r in zip(ts, rs):
        assert r["status"] == 0
        assert true_rel_residual(L, x, b) <= TOL * 1.0001


def test_admission_by_memory_budget(env):
    bd, _ = env
    L = I.laplacian3d(24)                       # 13,824 rows: a CG request needs ~0.6 MB
    with bd.Server(memory_budget=2 << 20) as S:   # room for three at a time
        mid = S.register(L)
        ts = [S.submit_cg(mid, I.uniform_pm1(20 + i, I.TAG_RHS, L.n), TOL) for i in range(8)]
        for t, _ in ts:
            assert S.wait(t)["status"] == 0
        st = S.stats()
    assert st["completed"] == 8
    assert 1 <= st["max_inflight_seen"] <= 3
    assert st["arena_used_max"] <= st["arena_capacity"]


def test_request_errors(env):
    bd, _ = env
    R = I.random_csr(50, 40, 0.1, 2)
    with bd.Server() as S:
        mid = S.register(R)
        with pytest.raises(bd.CbspmvError):
            S.submit_cg(mid, np.ones(40))                 # not square
        with pytest.raises(bd.CbspmvError):
            S.submit_spmv(mid + 5, np.ones(40))            # unknown matrix


def test_oversized_request_is_refused_at_submit(env):
    """A request whose workspace exceeds the whole memory budget is refused when it is
    submitted (it could never be admitted, and the arrival-order queue would hold every
    later request behind it); a small request after it still completes."""
    bd, torch = env
    big = I.laplacian3d(40)                      # 64,000 rows: a CG request needs ~2.8 MB
    small = I.random_csr(300, 200, 0.05, 4)
    with bd.Server(memory_budget=1 << 20) as S:
        mb, ms = S.register(big), S.register(small)
        with pytest.raises(bd.CbspmvError) as ei:
            S.submit_cg(mb, I.uniform_pm1(30, I.TAG_RHS, big.n), TOL)
        assert ei.value.status == 3               # CBSPMV_ERR_OOM
        x = I.vector_x(small.n, 31)
        t, y = S.submit_spmv(ms, x)
        r = S.wait(t, 60000)
        assert r["done"] and r["status"] == 0
        assert S.stats()["submitted"] == 1
    np.testing.assert_array_equal(y, solo_product(bd, torch, small, x))


def test_cg_limit_lets_products_pass(env):
    """max_inflight_cg = 1: solves run one at a time in arrival order while products
    submitted behind a waiting solve are admitted and finish first; every result equals the
    unlimited server's bit for bit (a request's result does not depend on the mix)."""
    bd, torch = env
    L = I.laplacian3d(16)
    bs = [I.uniform_pm1(90 + i, I.TAG_RHS, L.n) for i in range(3)]
    xs = [I.uniform_pm1(95 + i, I.TAG_X, L.n) for i in range(4)]
    res = {}
    for cap in (1, 0):
        with bd.Server(max_inflight_cg=cap) as S:
            mid = S.register(L)
            cg = [S.submit_cg(mid, b, TOL) for b in bs]
            pr = [S.submit_spmv(mid, x) for x in xs]
            rp = [S.wait(t) for t, _ in pr]
            rc = [S.wait(t) for t, _ in cg]
            res[cap] = ([y for _, y in pr], [x for _, x in cg])
            assert all(r["status"] == 0 for r in rp + rc)
            if cap == 1:
                # the products, submitted after three solves, finished before the last solve
                assert max(r["t_done"] for r in rp) < rc[-1]["t_done"]
                assert rc[0]["t_done"] <= rc[1]["t_done"] <= rc[2]["t_done"]
    for a, b in zip(res[1][0] + res[1][1], res[0][0] + res[0][1]):
        assert np.array_equal(a, b)
    for x, b in zip(res[1][1], bs):
        assert true_rel_residual(L, x, b) <= TOL * 1.0001


@pytest.mark.parametrize("inner_steps", [4, 16])
def test_oldest_first_quotas_keep_results(env, inner_steps):
    """cg_oldest_first: the oldest solve in its inner phase runs all inner_steps iterations
    per tick, the next half, the rest a quarter; every solve's result equals the same
    server's without the option bit for bit (iterations do not depend on how a tick groups
    them) and reaches the tolerance; products in the mix are unchanged."""
    bd, torch = env
    L1, L2 = I.laplacian3d(12), I.laplacian3d(16)
    bs = [I.uniform_pm1(110 + i, I.TAG_RHS, (L1 if i % 2 else L2).n) for i in range(5)]
    xs = [I.uniform_pm1(120 + i, I.TAG_X, L2.n) for i in range(3)]
    res = {}
    for oldest in (True, False):
        with bd.Server(inner_steps=inner_steps, cg_oldest_first=oldest) as S:
            m1, m2 = S.register(L1), S.register(L2)
            cg = [S.submit_cg(m1 if i % 2 else m2, b, TOL) for i, b in enumerate(bs)]
            pr = [S.submit_spmv(m2, x) for x in xs]
            rc = [S.wait(t) for t, _ in cg]
            rp = [S.wait(t) for t, _ in pr]
            assert all(r["status"] == 0 for r in rc + rp)
            res[oldest] = ([x for _, x in cg], [y for _, y in pr], [r["iterations"] for r in rc])
    for a, b in zip(res[True][0] + res[True][1], res[False][0] + res[False][1]):
        assert np.array_equal(a, b)
    assert res[True][2] == res[False][2]
    for i, (x, b) in enumerate(zip(res[True][0], bs)):
        assert true_rel_residual(L1 if i % 2 else L2, x, b) <= TOL * 1.0001
