"""GPU tests of cbspmv_update_values: a handle whose values were re-packed on the device
equals a fresh analysis of the new values bit for bit (exported values and products),
for every storage type, from host and from device arrays."""
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


CASES = {
    "fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
    "dense_70x45": lambda: I.random_csr(70, 45, 0.85, 6),          # Dense sub-blocks
    "rmat12": lambda: I.rmat(12, 16, seed=4),
    "laplace3d_10": lambda: I.laplacian3d(10),
}


def new_values(A, seed):
    return I.normal(seed, I.TAG_VAL, A.nnz) * 10.0 ** (np.arange(A.nnz) % 7 - 3)


@pytest.mark.parametrize("fmt", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("layout", [0, 1])
def test_update_equals_fresh_analysis(env, fmt, name, layout):
    bd, torch = env
    A = CASES[name]()
    v2 = new_values(A, 77)
    A2 = I.CSR(A.m, A.n, A.row_ptr, A.col, v2)
    vec = torch.float64 if fmt == "f64" else torch.float32
    x = I.vector_x(A.n, 5)
    with bd.BlockedMatrix(A, value_dtype=fmt, keep_value_map=True, record_layout=layout) as M, \
            bd.BlockedMatrix(A2, value_dtype=fmt, record_layout=layout) as F:
        M.update_values(v2)
        torch.cuda.synchronize()
        rp, col, val = M.export_csr()
        rpf, colf, valf = F.export_csr()
        assert np.array_equal(rp, rpf) and np.array_equal(col, colf)
        assert np.array_equal(val.view(np.uint64), valf.view(np.uint64))
        xd = torch.from_numpy(x).to(vec).cuda()
        y1 = torch.zeros(A.m, dtype=vec, device="cuda")
        y2 = torch.zeros(A.m, dtype=vec, device="cuda")
        M.run(xd, y1)
        F.run(xd, y2)
        assert torch.equal(y1, y2)
        M.check_device()
    if fmt == "f64":
        yref, s = oracle.spmv(A2, x)
        assert oracle.within_tolerance(y1.cpu().numpy(), yref, s)[0]


def test_update_from_device_array_and_repeatedly(env):
    bd, torch = env
    A = CASES["fem_small"]()
    x = I.vector_x(A.n, 6)
    xd = torch.from_numpy(x).cuda()
    with bd.BlockedMatrix(A, keep_value_map=True) as M:
        for rep in range(3):
            v = new_values(A, 100 + rep)
            M.update_values(torch.from_numpy(v).cuda())
            y = torch.zeros(A.m, dtype=torch.float64, device="cuda")
            M.run(xd, y)
            yref, s = oracle.spmv(I.CSR(A.m, A.n, A.row_ptr, A.col, v), x)
            assert oracle.within_tolerance(y.cpu().numpy(), yref, s)[0]
        M.check_device()


def test_update_needs_the_value_map(env):
    bd, _ = env
    A = CASES["laplace3d_10"]()
    with bd.BlockedMatrix(A) as M:
        with pytest.raises(bd.CbspmvError) as e:
            M.update_values(A.val)
        assert e.value.status == bd.CBSPMV_ERR_INVALID
