"""CPU tests of bench.py's host helpers: the row slices of the all-core oracle leg cover the
matrix exactly once and their products equal the single-threaded oracle's product."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2605_18515_gb300 import inputs as I  # noqa: E402


def test_row_slices_cover_rows_once_and_multiply_exactly():
    for A, parts in ((I.rmat(11, 16, seed=3), 7), (I.random_csr(301, 200, 0.05, 4), 16),
                     (I.random_csr(3, 50, 0.5, 5), 8)):
        x = I.vector_x(A.n, 6)
        sl = bench.row_slices(A, parts)
        assert sum(S.m for S in sl) == A.m and sum(S.row_ptr[-1] - S.row_ptr[0] for S in sl) == A.nnz
        y = np.concatenate([oracle.spmv(S, x)[0] for S in sl])
        assert np.array_equal(y, oracle.spmv(A, x)[0])


def test_allcore_oracle_reports_its_threads():
    A = I.random_csr(2000, 1500, 0.01, 7)
    gf, threads, sample = bench.oracle_allcore_gflops(A, I.vector_x(A.n, 8), target_s=0.2)
    assert gf > 0 and threads == len(os.sched_getaffinity(0)) and str(threads) in sample
