"""Pins for the oracle's restatement of the preprocessing (Sec. 3): hand-derived worked
examples (tests/golden), the thresholds of Sec. 3.3, the aggregation invariant of
Sec. 3.3.1, the storage model of Sec. 4.4.1, and the invariants of Algorithm 2."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import blocked as B
from paper_2605_18515_gb300 import inputs as I

FMT = {"COO": B.FMT_COO, "CSR": B.FMT_CSR, "DENSE": B.FMT_DENSE}


def example_32x48():
    r = [0, 1, 2, 3, 15, 16]
    c = [0, 17, 34, 35, 47, 0]
    rr, cc = np.meshgrid(np.arange(16, 32), np.arange(16, 32), indexing="ij")
    r = np.concatenate([r, rr.ravel()])
    c = np.concatenate([c, cc.ravel()])
    return I.csr_from_coo(32, 48, r, c, np.ones(r.size), sum_duplicates=False)


def test_worked_example_matches_hand_derivation():
    g = read_golden("blocked_example_32x48.txt")
    A = example_32x48()
    assert A.nnz == 262
    br, bc, cnt = B.plain_tiles(A)
    assert [f"{a},{b},{c}" for a, b, c in zip(br, bc, cnt)] == g["plain_tiles"]
    assert B.aggregation_decision(A) == bool(int(g["aggregated"][0]))
    S = B.blocked_structure(A)
    got = [f"{a},{b},{c},{k}" for a, b, c, k in zip(S.tile_brow, S.tile_bcol, S.tile_nnz,
                                                    [list(FMT)[f] for f in S.tile_fmt])]
    assert got == g["agg_tiles"]
    assert S.restore_cols.tolist() == [int(v) for v in g["restore_cols"]]
    assert S.cols_offset.tolist() == [int(v) for v in g["cols_offset"]]
    t0 = S.entry_tile == 0
    bytes0 = B.coord_byte(S.entry_lrow[t0], S.entry_lcol[t0])
    assert [f"0x{b:02x}" for b in bytes0] == g["coord_bytes_tile0"]
    S0 = B.blocked_structure(A, col_agg=0)
    assert [list(FMT)[f] for f in S0.tile_fmt] == g["noagg_formats"]
    st = B.storage_bytes(A.m, A.nnz, S0.tile_nnz.size, 2)
    assert st["csr"] == int(g["storage_csr"][0])
    assert st["bsr16"] == int(g["storage_bsr16"][0])
    assert st["cb_coo"] == int(g["storage_cb_coo"][0])


def test_coordinate_byte_roundtrip_and_nibble_order():
    rows, cols = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    b = B.coord_byte(rows, cols)
    assert b.min() == 0 and b.max() == 255 and np.unique(b).size == 256
    r2, c2 = B.decode_coord(b)
    assert np.array_equal(r2, rows) and np.array_equal(c2, cols)
    assert B.coord_byte(3, 5) == 0x53         # column in the high nibble (Algorithm 3)


@pytest.mark.parametrize("k,fmt", [(1, B.FMT_COO), (31, B.FMT_COO), (32, B.FMT_CSR),
                                   (128, B.FMT_CSR), (129, B.FMT_DENSE), (256, B.FMT_DENSE)])
def test_format_threshold_boundaries(k, fmt):
    # one 16x16 sub-block holding k nonzeros (row-major fill)
    idx = np.arange(k)
    A = I.csr_from_coo(16, 16, idx // 16, idx % 16, np.ones(k), sum_duplicates=False)
    S = B.blocked_structure(A)
    assert S.tile_nnz.tolist() == [k] and S.tile_fmt.tolist() == [fmt]


def diagonal_blocks(blocks):
    r, c = [], []
    for b, k in enumerate(blocks):
        idx = np.arange(k)
        r.append(16 * b + idx // 16)
        c.append(16 * b + idx % 16)
    n = 16 * len(blocks)
    return I.csr_from_coo(n, n, np.concatenate(r), np.concatenate(c), np.ones(sum(blocks)),
                          sum_duplicates=False)


def test_aggregation_threshold_is_strict():
    # 20 diagonal sub-blocks, 3 super-sparse (1 nnz) and 17 full: fraction 0.15 exactly -> off
    A = diagonal_blocks([1] * 3 + [256] * 17)
    assert B.super_sparse_fraction(A) == pytest.approx(0.15)
    assert not B.aggregation_decision(A)
    assert not B.blocked_structure(A).aggregated
    # 4 of 20 -> 0.2 > 0.15 -> on
    A = diagonal_blocks([1] * 4 + [256] * 16)
    assert B.aggregation_decision(A) and B.blocked_structure(A).aggregated
    # a sub-block with exactly 32 nonzeros is not super-sparse
    A = diagonal_blocks([32] * 20)
    assert B.super_sparse_fraction(A) == 0.0


def test_aggregated_blocks_hold_at_least_16_nonzeros():
    """Sec. 3.3.1: after aggregation every sub-block but the last of its block row has
    16 non-empty columns, hence at least 16 nonzeros."""
    for A in (I.random_csr(200, 3000, 0.004, 7), I.laplacian2d(32), I.rmat(10, 8, seed=3)):
        S = B.blocked_structure(A, col_agg=1)
        last = np.r_[S.tile_brow[1:] != S.tile_brow[:-1], True]
        assert np.all(S.tile_nnz[~last] >= 16)
        # restore_cols maps every entry back to its column
        r = B.entry_rows(A)
        back = S.restore_cols[S.cols_offset[r // 16] + 16 * S.tile_bcol[S.entry_tile] + S.entry_lcol]
        assert np.array_equal(back, A.col)


def test_alg2_hand_trace():
    g = read_golden("alg2_example.txt")
    order, end, loads = B.tb_load_balance([int(v) for v in g["nnz"]], int(g["warps_per_tb"][0]))
    assert end.tolist() == [int(v) for v in g["end"]]
    assert order.tolist() == [int(v) for v in g["order"]]
    assert loads.tolist() == [int(v) for v in g["tb_loads"]]


def test_alg2_invariants():
    nnz = (I.uniform01(9, 3, 1003) ** 4 * 256).astype(np.int64) + 1
    order, end, loads = B.tb_load_balance(nnz)
    assert np.array_equal(np.sort(order), np.arange(nnz.size))          # bijection
    ntb = (nnz.size + 7) // 8
    assert np.unique(end).size == nnz.size and end.min() >= 0 and end.max() < 8 * ntb
    assert np.bincount(end // 8).max() <= 8
    assert loads.sum() == nnz.sum()
    # LPT: except for the blocks that were filled last, loads differ by at most the largest item
    assert loads.max() - np.median(loads) <= nnz.max()


def test_storage_model_against_direct_count():
    A = I.random_csr(100, 90, 0.05, 12)
    S = B.blocked_structure(A, col_agg=0)
    nnzb = S.tile_nnz.size
    st = B.storage_bytes(A.m, A.nnz, nnzb, (A.m + 15) // 16)
    # direct count of a COO-only packing: 1 index byte + 8 value bytes per nonzero, and
    # blk_row, blk_col, nnz (int32), type (1 byte), vp (8 bytes) per sub-block
    assert st["cb_coo"] == nnzb * (4 + 4 + 4 + 1 + 8) + A.nnz * 9
    assert st["csr"] == A.row_ptr.size * 4 + A.col.size * 4 + A.val.size * 8


def test_histogram_bins():
    coarse, fine = B.nnz_histogram([1, 8, 9, 16, 17, 32, 33, 64, 65, 256])
    assert coarse.tolist() == [6, 2, 1, 0, 0, 0, 0, 1]
    assert fine.tolist() == [2, 2, 1, 1]
