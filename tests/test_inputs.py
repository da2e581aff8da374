"""Pins for the seeded input generators (shared by the oracle and the CUDA path)."""
import numpy as np

from conftest import read_golden
from paper_2605_18515_gb300 import inputs as I


def test_splitmix64_published_vector():
    g = read_golden("splitmix64.txt")
    want = [int(v, 16) for v in g["seed0_first"]]
    got = [I._mix_scalar((k + 1) * I.GAMMA) for k in range(3)]
    assert got == want
    # the vectorised stream equals the scalar definition
    key = I.stream_key(7, I.TAG_X)
    z = I.draws_u64(7, I.TAG_X, 5, 4)
    assert [int(v) for v in z] == [I._mix_scalar(key + (k + 6) * I.GAMMA) for k in range(4)]


def is_canonical(A):
    rp, c = A.row_ptr, A.col.astype(np.int64)
    if rp[0] != 0 or np.any(np.diff(rp) < 0) or rp[-1] != c.size:
        return False
    if c.size and (c.min() < 0 or c.max() >= A.n):
        return False
    rows = np.repeat(np.arange(A.m), np.diff(rp))
    same = rows[1:] == rows[:-1]
    return bool(np.all(np.diff(c)[same] > 0))


def test_laplacian_sizes():
    A = I.laplacian2d(64)
    assert (A.m, A.n, A.nnz) == (4096, 4096, 5 * 4096 - 4 * 64) and is_canonical(A)
    B = I.laplacian3d(8)
    assert B.nnz == 7 * 512 - 6 * 64 and is_canonical(B)


def test_uniform_ranges_and_determinism():
    u = I.uniform01(1, 2, 100000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
    v = I.uniform_pm1(1, 2, 100000)
    assert np.array_equal(v, 2 * u - 1)
    z = I.normal(3, 4, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert np.array_equal(I.vector_x(1000, 5), I.vector_x(1000, 5))
    assert not np.array_equal(I.vector_x(1000, 5), I.vector_x(1000, 6))


def test_fem_block_band_small():
    A = I.fem_block_band(n_rows=3000, n_block_rows=1000, half_band=50, seed=1)
    assert is_canonical(A)
    # block structure: every row of a 3-row block row has the same column list
    for I0 in (0, 17, 999):
        r0 = 3 * I0
        cols0 = A.col[A.row_ptr[r0]:A.row_ptr[r0 + 1]]
        for r in range(r0, min(r0 + 3, A.m)):
            assert np.array_equal(A.col[A.row_ptr[r]:A.row_ptr[r + 1]], cols0)
        bcols = np.unique(cols0 // 3)
        assert I0 in bcols and np.all(np.abs(bcols - I0) <= 50) and bcols.size <= 27
    # interior block rows have exactly 27 blocks -> 81 nonzeros per row
    assert np.diff(A.row_ptr)[150] == 81


def test_fem_clipped_last_block():
    A = I.fem_block_band(n_rows=3001, n_block_rows=1001, half_band=20, seed=1)
    assert A.m == 3001 and is_canonical(A)
    last = A.col[A.row_ptr[-2]:A.row_ptr[-1]]
    assert last.max() <= 3000


def test_rmat_small():
    A = I.rmat(10, 8, seed=2)
    assert A.m == 1024 and is_canonical(A) and 0 < A.nnz <= 8 * 1024
    deg = np.diff(A.row_ptr)
    assert deg[0] > deg[-1]                   # quadrant a biases toward low indices
    assert np.array_equal(A.col, I.rmat(10, 8, seed=2).col)
