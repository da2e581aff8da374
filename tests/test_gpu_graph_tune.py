"""GPU tests of CUDA-graph captured batched products and of the autotuned analysis: graph
replays equal direct batched runs bit for bit (and follow new X contents); the tuned
handle computes the same product within the oracle tolerance and reports its candidates."""
import numpy as np
import pytest

import oracle
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


def test_graph_replays_batched_products(env):
    bd, torch = env
    As = [I.laplacian3d(10), I.random_csr(333, 517, 0.2, 11), I.rmat(12, 16, seed=4)]
    Ms = bd.analyze_batched(As)
    try:
        Xs = [torch.from_numpy(I.vector_x(A.n, 60 + i)).cuda() for i, A in enumerate(As)]
        Ys = [torch.zeros(A.m, dtype=torch.float64, device="cuda") for A in As]
        Yd = [torch.zeros(A.m, dtype=torch.float64, device="cuda") for A in As]
        with bd.Graph(Ms, Xs, Ys, [1.0, -2.0, 0.5], [0.0, 0.0, 0.0]) as G:
            for rep in range(3):
                for i, A in enumerate(As):          # new x contents before each replay
                    Xs[i].copy_(torch.from_numpy(I.vector_x(A.n, 100 * rep + i)))
                G.launch()
                bd.run_batched(Ms, Xs, Yd, [1.0, -2.0, 0.5], [0.0, 0.0, 0.0])
                torch.cuda.synchronize()
                for i, A in enumerate(As):
                    assert torch.equal(Ys[i], Yd[i])
                    x = Xs[i].cpu().numpy()
                    yref, s = oracle.spmv(A, x, [1.0, -2.0, 0.5][i])
                    assert oracle.within_tolerance(Ys[i].cpu().numpy(), yref, s, [1.0, -2.0, 0.5][i])[0]
        for M in Ms:
            M.check_device()
    finally:
        for M in Ms:
            M.close()


@pytest.mark.parametrize("name", ["fem_small", "rmat12"])
@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_tuned_analysis(env, name, dtype):
    bd, torch = env
    if dtype != "f64":
        pytest.skip("reduced types: covered by test_tuned_analysis_reduced_type")
    A = {"fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
         "rmat12": lambda: I.rmat(12, 16, seed=4)}[name]()
    M, rep = bd.analyze_tuned(A, reps=5)
    with M:
        # FP64: aggregation side, two lane unit sizes, the record layout (then its own axes
        # when it wins)
        assert 4 <= rep["n_tried"] <= 16
        assert any(t["record_layout"] == 1 for t in rep["tried"])
        assert M.stats()["lane_layout"] == (rep["best"]["record_layout"] == 0)
        assert rep["best_ms"] <= rep["default_ms"] and rep["best_ms"] == min(t["ms"] for t in rep["tried"])
        x = I.vector_x(A.n, 12)
        yd = torch.zeros(A.m, dtype=torch.float64, device="cuda")
        M.run(torch.from_numpy(x).cuda(), yd)
        yref, s = oracle.spmv(A, x)
        assert oracle.within_tolerance(yd.cpu().numpy(), yref, s)[0]
        st = M.stats()
        assert st["aggregated"] == (rep["best"]["col_agg"] == 1 or
                                    (rep["best"]["col_agg"] == -1 and st["super_sparse_fraction"] > 0.15))


def test_tuned_analysis_reduced_type(env):
    """BF16 values: aggregation, the lane-stream unit sizes, the record layout against the
    default lane streams, then, when the records win, their axes (unit sizes and the format
    thresholds); the tuned
    handle's product stays within the FP32 bound of the stored-value product."""
    from oracle import lowprec as L
    bd, torch = env
    A = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    M, rep = bd.analyze_tuned(A, reps=5, value_dtype="bf16")
    with M:
        assert 5 <= rep["n_tried"] <= 16
        assert any(t["record_layout"] == 1 for t in rep["tried"]) and rep["tried"][0]["record_layout"] == 0
        assert M.stats()["lane_layout"] == (rep["best"]["record_layout"] == 0)
        assert rep["best_ms"] == min(t["ms"] for t in rep["tried"])
        x = I.vector_x(A.n, 13).astype(np.float32)
        yd = torch.zeros(A.m, dtype=torch.float32, device="cuda")
        M.run(torch.from_numpy(x).cuda(), yd)
        y_ref, s = oracle.spmv(L.stored_matrix(A, "bf16"), x.astype(np.float64))
        assert L.within_bound(yd.cpu().numpy(), y_ref, s, L.fp32_bound(A))[0]
