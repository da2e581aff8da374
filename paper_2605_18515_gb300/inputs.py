"""Seeded synthetic inputs for the blocked SpMV: matrices in canonical CSR and dense vectors.

This module only *builds inputs*. It holds none of the SpMV method's arithmetic (no
tiling, no aggregation, no products): both the CPU oracle and the CUDA path consume
its arrays, so neither depends on the other.

Random numbers come from one counter-based generator, SplitMix64 (G. Steele, D. Lea,
C. Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the k-th
64-bit draw of a stream is ``mix(key + (k + 1) * GAMMA)`` (mod 2**64) with the
published finaliser ``mix`` and golden-ratio increment ``GAMMA``. A stream key is
``mix(seed * GAMMA ^ tag)`` where ``tag`` names the stream ("x", "val", ...), so every
array can be regenerated independently, in any order, on any machine.

Conversions:
  * uniform in [0, 1): top 53 bits times 2**-53;
  * uniform in [-1, 1): ``2u - 1``;
  * N(0, 1): Box-Muller ``sqrt(-2 ln u1) * cos(2 pi u2)`` with u1 in (0, 1], u2 in [0, 1)
    taken from draws 2k and 2k+1 of the stream.

Workload recipes (sizes of the paper's evaluation stand-ins; the paper's SuiteSparse
matrices, Sec. 4.1, are not available, so these synthetic families stand in for them):
  * ``laplacian2d(g)``: 5-point stencil on a g x g grid, natural ordering, 4 on the
    diagonal, -1 off it; g = 64 gives 4096 rows and 20,224 nonzeros.
  * ``laplacian3d(g)``: 7-point stencil on a g^3 grid, 6 / -1.
  * ``fem_block_band``: rows grouped in 3-row block rows; each block row holds its
    diagonal 3x3 block plus 26 off-diagonal 3x3 blocks, one drawn uniformly from each of
    26 equal strata of the offsets {-W..-1, 1..W} (W = 1000 block columns, so the band
    spans 2,000 block columns and the 26 offsets are distinct and sorted); blocks falling
    outside the matrix are dropped and the last block row/column is clipped to the
    matrix edge. Values N(0, 1) by CSR position.
  * ``rmat``: R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with 2**scale vertices and
    edge_factor * 2**scale edge samples, probabilities (a, b, c, d); each level picks a
    quadrant from a 21-bit uniform (three levels share one 64-bit draw); no noise, no
    vertex permutation, self loops kept, duplicate (row, col) samples summed. Each
    sample carries a U[-1, 1) value.
"""
from __future__ import annotations

import dataclasses
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

# stream tags
TAG_X = 1
TAG_VAL = 2
TAG_STRUCT = 3
TAG_Y = 4
TAG_RHS = 5


def _mix_scalar(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def stream_key(seed: int, tag: int) -> int:
    return _mix_scalar(((seed * GAMMA) & _MASK) ^ tag)


def _mix_inplace(z: np.ndarray) -> np.ndarray:
    t = np.empty_like(z)
    np.right_shift(z, np.uint64(30), out=t)
    np.bitwise_xor(z, t, out=z)
    np.multiply(z, np.uint64(_M1), out=z)
    np.right_shift(z, np.uint64(27), out=t)
    np.bitwise_xor(z, t, out=z)
    np.multiply(z, np.uint64(_M2), out=z)
    np.right_shift(z, np.uint64(31), out=t)
    np.bitwise_xor(z, t, out=z)
    return z


def draws_u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of stream (seed, tag) as uint64."""
    key = np.uint64(stream_key(seed, tag))
    with np.errstate(over="ignore"):
        z = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        np.multiply(z, np.uint64(GAMMA), out=z)
        np.add(z, key, out=z)
        return _mix_inplace(z)


def uniform01(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    z = draws_u64(seed, tag, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    return 2.0 * uniform01(seed, tag, count, start) - 1.0


def normal(seed: int, tag: int, count: int) -> np.ndarray:
    z = draws_u64(seed, tag, 0, 2 * count)
    u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass
class CSR:
    """Canonical CSR: int64 row_ptr (m+1), int32 col (nnz, strictly increasing per row),
    float64 val (nnz)."""
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self) -> np.ndarray:
        """Row index of every stored entry."""
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.row_ptr))


def csr_from_coo(m: int, n: int, r: np.ndarray, c: np.ndarray, v: np.ndarray,
                 name: str = "", sum_duplicates: bool = True) -> CSR:
    """Sort (r, c) row-major; duplicate coordinates are summed in sample order."""
    key = r.astype(np.int64) * n + c.astype(np.int64)
    if sum_duplicates:
        uk, inv = np.unique(key, return_inverse=True)
        vals = np.bincount(inv.ravel(), weights=v, minlength=uk.size)
    else:
        order = np.argsort(key, kind="stable")
        uk = key[order]
        vals = v[order]
        if uk.size > 1 and np.any(uk[1:] == uk[:-1]):
            raise ValueError("duplicate coordinates")
    rows = uk // n
    cols = (uk % n).astype(np.int32)
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(m, n, row_ptr, cols, np.ascontiguousarray(vals, dtype=np.float64), name)


def laplacian2d(g: int = 64) -> CSR:
    idx = np.arange(g * g, dtype=np.int64)
    p, q = idx // g, idx % g
    rs, cs, vs = [], [], []
    for dp, dq, w in ((-1, 0, -1.0), (0, -1, -1.0), (0, 0, 4.0), (0, 1, -1.0), (1, 0, -1.0)):
        ok = (p + dp >= 0) & (p + dp < g) & (q + dq >= 0) & (q + dq < g)
        rs.append(idx[ok]); cs.append((p[ok] + dp) * g + q[ok] + dq); vs.append(np.full(ok.sum(), w))
    return csr_from_coo(g * g, g * g, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs),
                        name=f"laplacian2d_{g}", sum_duplicates=False)


def laplacian3d(g: int) -> CSR:
    N = g * g * g
    idx = np.arange(N, dtype=np.int64)
    i, j, k = idx // (g * g), (idx // g) % g, idx % g
    rs, cs, vs = [], [], []
    for di, dj, dk, w in ((-1, 0, 0, -1.0), (0, -1, 0, -1.0), (0, 0, -1, -1.0), (0, 0, 0, 6.0),
                          (0, 0, 1, -1.0), (0, 1, 0, -1.0), (1, 0, 0, -1.0)):
        ok = ((i + di >= 0) & (i + di < g) & (j + dj >= 0) & (j + dj < g)
              & (k + dk >= 0) & (k + dk < g))
        rs.append(idx[ok]); cs.append(((i[ok] + di) * g + j[ok] + dj) * g + k[ok] + dk)
        vs.append(np.full(ok.sum(), w))
    return csr_from_coo(N, N, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs),
                        name=f"laplacian3d_{g}", sum_duplicates=False)


def fem_block_band(n_rows: int = 1_048_576, n_block_rows: int = 349_526, half_band: int = 1000,
                   offdiag: int = 26, bs: int = 3, seed: int = 1) -> CSR:
    """Block-structured FEM-like matrix (see module docstring for the recipe)."""
    nb = n_block_rows
    m = n = n_rows
    if 2 * half_band < offdiag or offdiag % 2:
        raise ValueError("need an even number of strata, each holding at least one offset")
    # strata of the sorted offset list {-W..-1, 1..W}
    offs_all = np.concatenate([np.arange(-half_band, 0), np.arange(1, half_band + 1)])
    L = offs_all.size
    lo = (np.arange(offdiag) * L) // offdiag
    hi = (np.arange(1, offdiag + 1) * L) // offdiag
    u = uniform01(seed, TAG_STRUCT, nb * offdiag).reshape(nb, offdiag)
    pick = lo[None, :] + np.minimum((u * (hi - lo)[None, :]).astype(np.int64), (hi - lo - 1)[None, :])
    offs = offs_all[pick]                                   # (nb, 26) sorted ascending
    I = np.arange(nb, dtype=np.int64)[:, None]
    split = np.searchsorted(offs_all[lo], 0)                # strata entirely below zero come first
    J = np.concatenate([I + offs[:, :split], I, I + offs[:, split:]], axis=1)  # (nb, 27) sorted
    jvalid = (J >= 0) & (J < nb)
    # columns of each block row: bs per block column, clipped to n
    cols = (J[:, :, None] * bs + np.arange(bs)[None, None, :]).reshape(nb, -1)   # (nb, 27*bs)
    cvalid = np.repeat(jvalid, bs, axis=1) & (cols < n)
    per_brow = cvalid.sum(axis=1)                           # nnz per row within block row I
    rows_in_brow = np.minimum(bs, m - np.arange(nb) * bs)   # last block row may be clipped
    counts = np.repeat(per_brow, rows_in_brow)
    assert counts.size == m
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    flat_cols = cols[cvalid].astype(np.int32)               # per block row, concatenated
    brow_start = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(per_brow, out=brow_start[1:])
    # each row of block row I repeats I's column list
    row_brow = np.repeat(np.arange(nb), rows_in_brow)
    nnz = int(row_ptr[-1])
    pos_in_row = np.arange(nnz, dtype=np.int64) - np.repeat(row_ptr[:-1], counts)
    col = flat_cols[np.repeat(brow_start[row_brow], counts) + pos_in_row]
    val = normal(seed, TAG_VAL, nnz)
    return CSR(m, n, row_ptr, col, val, name="fem_block_band")


def rmat(scale: int = 21, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 2) -> CSR:
    """R-MAT graph as a CSR matrix (see module docstring)."""
    nv = 1 << scale
    ne = edge_factor * nv
    row = np.zeros(ne, dtype=np.int64)
    col = np.zeros(ne, dtype=np.int64)
    ta, tab, tabc = a, a + b, a + b + c
    groups = (scale + 2) // 3
    mask21 = np.uint64((1 << 21) - 1)
    for gi in range(groups):
        z = draws_u64(seed, TAG_STRUCT, gi * ne, ne)
        for s in range(3):
            level = gi * 3 + s
            if level >= scale:
                break
            u = ((z >> np.uint64(21 * s)) & mask21).astype(np.float64) * (2.0 ** -21)
            bit = np.int64(1 << (scale - 1 - level))
            rbit = u >= tab                      # quadrants c, d set the row bit
            cbit = ((u >= ta) & (u < tab)) | (u >= tabc)   # quadrants b, d set the column bit
            row += rbit * bit
            col += cbit * bit
        del z
    v = uniform_pm1(seed, TAG_VAL, ne)
    return csr_from_coo(nv, nv, row, col, v, name=f"rmat_s{scale}")


def random_csr(m: int, n: int, density: float, seed: int, zero_rows: bool = True) -> CSR:
    """Small random canonical CSR (test helper): each (i, j) kept with prob. density."""
    u = uniform01(seed, TAG_STRUCT, m * n).reshape(m, n)
    keep = u < density
    if zero_rows and m > 2:
        keep[m // 3, :] = False
    r, c = np.nonzero(keep)
    v = uniform_pm1(seed, TAG_VAL, r.size)
    return csr_from_coo(m, n, r, c, v, name=f"random_{m}x{n}_{density}", sum_duplicates=False)


def vector_x(n: int, seed: int, k: int = 1) -> np.ndarray:
    """Dense right-hand side(s) U[-1, 1): shape (n,) for k == 1 else (k, n) row-major."""
    x = uniform_pm1(seed, TAG_X, n * k)
    return x if k == 1 else x.reshape(k, n)


# The configurations of the evaluation, by name.
def config_matrix(name: str) -> tuple[CSR, np.ndarray]:
    if name == "laplace2d_64":
        A = laplacian2d(64)
        return A, vector_x(A.n, 0)
    if name == "fem3x3_band_1m":
        A = fem_block_band(seed=1)
        return A, vector_x(A.n, 1)
    if name == "fem3x3_band_256k":
        # quarter-size profiling case of the FEM family (packed stream still > L2)
        A = fem_block_band(n_rows=262_144, n_block_rows=87_382, seed=1)
        return A, vector_x(A.n, 1)
    if name == "rmat_s21":
        A = rmat(21, 16, seed=2)
        return A, vector_x(A.n, 2)
    if name == "rmat_s19":
        # smaller profiling case of the R-MAT family (packed stream still > L2)
        A = rmat(19, 16, seed=2)
        return A, vector_x(A.n, 2)
    raise KeyError(name)


def isolated_entries_block_row(tiles: int = 20, rows_with_two: int = 11, seed: int = 9):
    """One block row of `tiles` 16x16 tiles (16 rows, 16 * tiles columns) whose first
    `rows_with_two` rows hold two isolated entries per tile (tile columns 0 and 8) and the
    other rows one (tile column 4): pieces of one or two entries, N(0,1) values."""
    r, c = [], []
    for t in range(tiles):
        for row in range(16):
            for cc in ((0, 8) if row < rows_with_two else (4,)):
                r.append(row)
                c.append(16 * t + cc)
    r, c = np.array(r, dtype=np.int64), np.array(c, dtype=np.int64)
    return csr_from_coo(16, 16 * tiles, r, c, normal(seed, TAG_VAL, r.size))
