"""Randomised CPU round trips of the host analysis: for seeded random matrices (shapes,
densities, empty rows and columns, dense blocks) and option combinations (aggregation
forced or decided, format thresholds, unit sizes, load balance, value types, value map),
the blocked structure equals the oracle's restatement and the packed format decodes to
the input bit for bit (FP64) or to the oracle's rounding of it (reduced types)."""
import numpy as np
import pytest

from oracle import blocked as B
from oracle import lowprec as L
from paper_2605_18515_gb300 import build, inputs as I


@pytest.fixture(scope="module")
def bd():
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding


def random_matrix(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 700)), int(rng.integers(1, 700))
    kind = seed % 3
    if kind == 0:                                   # uniform random
        A = I.random_csr(m, n, float(rng.uniform(0.001, 0.4)), seed)
    elif kind == 1:                                 # dense 16x16-ish blocks on a sparse background
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
        A = I.csr_from_coo(m, n, key // n, key % n, I.uniform_pm1(seed, 2, key.size), sum_duplicates=False)
    else:                                           # power law
        A = I.rmat(int(rng.integers(6, 10)), 16, seed=seed)
    return A


@pytest.mark.parametrize("seed", range(36))
def test_random_roundtrip(bd, seed):
    rng = np.random.default_rng(1000 + seed)
    A = random_matrix(seed)
    th1 = int(rng.choice([0, 8, 32, 64]))
    th2 = int(rng.choice([th1, 128, 200, 256])) if th1 <= 128 else 256
    th2 = max(th1, th2)
    opts = dict(col_agg=int(rng.choice([-1, 0, 1])), th1=th1, th2=th2,
                unit_work=int(rng.choice([0, 64, 300, 1024])), load_balance=bool(rng.integers(2)),
                keep_value_map=bool(rng.integers(2)))
    fmt = str(rng.choice(["f64", "f64", "f32", "bf16", "f16"]))
    with bd.BlockedMatrix(A, device=-1, value_dtype=fmt, **opts) as M:
        rp, col, val = M.export_csr()
        got = M.export_blocked()
        st = M.stats()
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    ref = A.val if fmt == "f64" else L.round_to_format(A.val, fmt)
    assert np.array_equal(val.view(np.uint64), ref.view(np.uint64))
    S = B.blocked_structure(A, th1=th1, th2=th2, col_agg=opts["col_agg"])
    assert got["aggregated"] == S.aggregated
    assert np.array_equal(got["blk_row"], S.tile_brow) and np.array_equal(got["blk_col"], S.tile_bcol)
    assert np.array_equal(got["nnz"], S.tile_nnz) and np.array_equal(got["type"], S.tile_fmt)
    # every unit is scheduled in exactly one mode
    assert st["n_entry_mode_units"] + st["n_xseq_units"] <= st["n_units"]
