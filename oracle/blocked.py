"""The preprocessing of Sec. 3, restated step by step in the paper's order -- test
infrastructure only (see ``oracle/__init__.py``).

Each function follows one passage:
  * 2D structure, Sec. 3.1: uniform 16x16 sub-blocks, high-level COO metadata
    (block row, block column, nnz, format) per non-empty sub-block.
  * Coordinate compression, Sec. 3.2: the in-block (row, col) pair of 4-bit indices in one
    byte; the decoding of Algorithm 3 reads the row from the low nibble and the column from
    the high nibble.
  * Column aggregation, Sec. 3.3.1: inside each 16-row block row, columns without any
    nonzero are removed and the remaining ones are shifted left, then cut into 16-wide
    sub-blocks again; ``restore_cols`` maps an aggregated column back to the original
    column and ``cols_offset`` gives the start of each block row's list. Applied only if
    the fraction of "super-sparse" sub-blocks (fewer than 32 nonzeros) exceeds th_0 = 0.15.
  * Format selection, Sec. 3.3.2: COO below th_1 = 32 nonzeros, Dense above th_2 = 128,
    CSR in between.
  * Storage model, Sec. 4.4.1: closed-form byte counts for CSR, BSR-16 and CB (all COO).
  * Thread-block load balance, Sec. 3.4, Algorithm 2: sub-blocks sorted by nnz, then
    handed one by one to the least-loaded thread block (a min-heap of (load, id)) until it
    holds 8 sub-blocks (one per warp); slot = tb_id * 8 + warps; metadata re-sorted by slot.

Readings where the paper is silent or garbled (each is also listed in the design notes):
  * the aggregation flag is matrix-wide and compares the fraction strictly (> th_0);
  * the aggregated x index is cols_offset[block row] + 16 * (aggregated block column) +
    in-block column (Algorithm 3 prints only cols_offset[block row] + column);
  * a sub-block with exactly 32 or exactly 128 nonzeros is CSR ("less than th_1",
    "more than th_2");
  * Algorithm 2 sorts by nnz in descending order (longest-processing-time first), with a
    stable sort and heap ties broken by thread-block id.
"""
from __future__ import annotations

import dataclasses
import heapq

import numpy as np

BLK = 16
TH0 = 0.15
TH1 = 32
TH2 = 128
WARPS_PER_TB = 8
FMT_COO, FMT_CSR, FMT_DENSE = 0, 1, 2


def coord_byte(row, col):
    """Sec. 3.2: two 4-bit in-block indices in one byte (row low nibble, col high nibble)."""
    return (np.asarray(row) & 15) | ((np.asarray(col) & 15) << 4)


def decode_coord(b):
    """Algorithm 3: row = b & 15, col = b >> 4."""
    b = np.asarray(b)
    return b & 15, b >> 4


def entry_rows(A) -> np.ndarray:
    return np.repeat(np.arange(A.m, dtype=np.int64), np.diff(A.row_ptr))


def plain_tiles(A):
    """Sec. 3.1 without aggregation: (block row, block col) of every entry and the nnz of
    each non-empty 16x16 sub-block, sub-blocks listed in row-major order."""
    r = entry_rows(A)
    c = A.col.astype(np.int64)
    nbc = (A.n + BLK - 1) // BLK
    key = (r // BLK) * nbc + c // BLK
    uk, counts = np.unique(key, return_counts=True)
    return uk // nbc, uk % nbc, counts


def super_sparse_fraction(A, th1: int = TH1) -> float:
    """Share of non-empty 16x16 sub-blocks holding fewer than th_1 nonzeros (Sec. 3.3.1)."""
    _, _, counts = plain_tiles(A)
    return float(np.mean(counts < th1)) if counts.size else 0.0


def aggregation_decision(A, th0: float = TH0, th1: int = TH1) -> bool:
    return super_sparse_fraction(A, th1) > th0


def column_aggregation(A):
    """Sec. 3.3.1. Returns (restore_cols int32, cols_offset int64 of length nbr+1, the
    aggregated column of every entry)."""
    r = entry_rows(A)
    br = r // BLK
    c = A.col.astype(np.int64)
    nbr = (A.m + BLK - 1) // BLK
    key = br * A.n + c
    uk, inv = np.unique(key, return_inverse=True)     # distinct (block row, column), sorted
    ubr = uk // A.n
    restore_cols = (uk % A.n).astype(np.int32)
    per_br = np.bincount(ubr, minlength=nbr)
    cols_offset = np.zeros(nbr + 1, dtype=np.int64)
    np.cumsum(per_br, out=cols_offset[1:])
    agg_col = np.arange(uk.size, dtype=np.int64)[inv.ravel()] - cols_offset[br]
    return restore_cols, cols_offset, agg_col


def select_format(nnz, th1: int = TH1, th2: int = TH2):
    """Sec. 3.3.2: COO if nnz < th_1, Dense if nnz > th_2, CSR otherwise."""
    nnz = np.asarray(nnz)
    return np.where(nnz < th1, FMT_COO, np.where(nnz > th2, FMT_DENSE, FMT_CSR)).astype(np.uint8)


@dataclasses.dataclass
class Blocked:
    aggregated: bool
    tile_brow: np.ndarray      # int64, row-major order
    tile_bcol: np.ndarray      # int64 (aggregated block column when aggregated)
    tile_nnz: np.ndarray       # int64
    tile_fmt: np.ndarray       # uint8
    restore_cols: np.ndarray   # int32 (empty when not aggregated)
    cols_offset: np.ndarray    # int64, nbr+1 (empty when not aggregated)
    entry_tile: np.ndarray     # int64 tile id of every CSR entry
    entry_lrow: np.ndarray     # in-block row of every CSR entry
    entry_lcol: np.ndarray     # in-block (aggregated) column of every CSR entry


def blocked_structure(A, th0: float = TH0, th1: int = TH1, th2: int = TH2,
                      col_agg: int = -1) -> Blocked:
    """Sec. 3 overview: decide on column aggregation (col_agg -1 = by th_0, 0 = off,
    1 = on), aggregate, form the 2D structure, then select a format per sub-block."""
    aggregated = aggregation_decision(A, th0, th1) if col_agg < 0 else bool(col_agg)
    r = entry_rows(A)
    br = r // BLK
    if aggregated:
        restore_cols, cols_offset, acol = column_aggregation(A)
    else:
        restore_cols = np.zeros(0, dtype=np.int32)
        cols_offset = np.zeros(0, dtype=np.int64)
        acol = A.col.astype(np.int64)
    bc = acol // BLK
    nbc = max((A.n + BLK - 1) // BLK, int(bc.max()) + 1 if bc.size else 1)
    key = br * nbc + bc
    uk, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    return Blocked(aggregated, uk // nbc, uk % nbc, counts.astype(np.int64), select_format(counts, th1, th2),
                   restore_cols, cols_offset, inv.ravel().astype(np.int64), r % BLK, acol % BLK)


def storage_bytes(m: int, nnz: int, nnzb: int, blk_m: int) -> dict:
    """Sec. 4.4.1 storage model: int32 positions, FP64 values, 16x16 blocks."""
    return {
        "csr": (m + 1) * 4 + nnz * 4 + nnz * 8,
        "bsr16": 256 * 8 * nnzb + (blk_m + 1) * 4 + nnzb * 4,
        "cb_coo": nnzb * (4 + 4 + 4 + 1 + 8) + nnz * (1 + 8),
    }


def tb_load_balance(nnz_per_blk, warps_per_tb: int = WARPS_PER_TB):
    """Algorithm 2. Returns (order, end, tb_loads): ``order[i]`` is the original index of
    the sub-block placed at position i after the final re-sort, ``end[j]`` the slot
    (tb_id * warps_per_tb + warp) given to original sub-block j, and the nnz each thread
    block received. Pure-Python heap loop: small inputs only."""
    nnz = np.asarray(nnz_per_blk, dtype=np.int64)
    nblk = nnz.size
    ntb = (nblk + warps_per_tb - 1) // warps_per_tb
    ori_sorted = np.argsort(-nnz, kind="stable")          # descending nnz
    heap = [(0, tb, 0) for tb in range(ntb)]               # (loads, tb_id, warps)
    heapq.heapify(heap)
    end = np.empty(nblk, dtype=np.int64)
    for j in ori_sorted:
        loads, tb, warps = heapq.heappop(heap)
        end[j] = tb * warps_per_tb + warps
        loads += int(nnz[j])
        warps += 1
        if warps < warps_per_tb:
            heapq.heappush(heap, (loads, tb, warps))
    order = np.argsort(end, kind="stable")
    tb_loads = np.bincount(end // warps_per_tb, weights=nnz, minlength=ntb).astype(np.int64)
    return order, end, tb_loads


def nnz_histogram(tile_nnz):
    """The sub-block histogram of Sec. 2.2 (Fig. 3): eight bins of 32 (1-32 ... 225-256)
    and the 1-32 bin split into 1-8, 9-16, 17-24, 25-32."""
    t = np.asarray(tile_nnz)
    coarse = np.bincount(np.clip((t - 1) // 32, 0, 7), minlength=8)
    small = t[t <= 32]
    fine = np.bincount(np.clip((small - 1) // 8, 0, 3), minlength=4)
    return coarse, fine
