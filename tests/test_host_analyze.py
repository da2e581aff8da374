"""CPU tests of the library's host analysis through the C ABI (host-only handles, no GPU):
the blocked structure must equal the oracle's restatement of Sec. 3 exactly, the packed
format must round-trip to the input CSR bit for bit, the load balance must keep its
invariants and bad input must come back as status codes."""
import ctypes

import numpy as np
import pytest

from oracle import blocked as B
from paper_2605_18515_gb300 import build, inputs as I


@pytest.fixture(scope="module")
def bd():
    build.build()
    from paper_2605_18515_gb300 import binding
    return binding


def host(bd, A, **kw):
    return bd.BlockedMatrix(A, device=-1, **kw)


CASES = {
    "laplace2d_64": lambda: I.laplacian2d(64),
    "laplace3d_9": lambda: I.laplacian3d(9),
    "random_ragged": lambda: I.random_csr(203, 157, 0.07, 5),
    "random_dense": lambda: I.random_csr(70, 45, 0.8, 6),
    "rmat10": lambda: I.rmat(10, 16, seed=4),
    "fem_small": lambda: I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
    "one_row": lambda: I.random_csr(1, 300, 0.5, 7),
    "one_col": lambda: I.random_csr(300, 1, 0.5, 8),
}


def assert_same_structure(bd, A, M, col_agg=-1, th1=32, th2=128, th0=0.15):
    S = B.blocked_structure(A, th0=th0, th1=th1, th2=th2, col_agg=col_agg)
    got = M.export_blocked()
    assert got["aggregated"] == S.aggregated
    assert np.array_equal(got["blk_row"], S.tile_brow)
    assert np.array_equal(got["blk_col"], S.tile_bcol)
    assert np.array_equal(got["nnz"], S.tile_nnz)
    assert np.array_equal(got["type"], S.tile_fmt)
    if S.aggregated:
        assert np.array_equal(got["cols_offset"], S.cols_offset)
        assert np.array_equal(got["restore_cols"], S.restore_cols)
    st = M.stats()
    assert st["n_tiles"] == S.tile_nnz.size
    assert st["super_sparse_fraction"] == pytest.approx(B.super_sparse_fraction(A, th1), abs=0)
    coarse, fine = B.nnz_histogram(S.tile_nnz)
    assert st["hist_coarse"] == coarse.tolist() and st["hist_fine"] == fine.tolist()


def assert_roundtrip(M, A):
    rp, col, val = M.export_csr()
    assert np.array_equal(rp, A.row_ptr)
    assert np.array_equal(col, A.col)
    assert np.array_equal(val.view(np.uint64), A.val.view(np.uint64))   # bit-exact


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("col_agg", [-1, 0, 1])
@pytest.mark.parametrize("layout", ["lanes", "records"])
def test_structure_and_roundtrip(bd, name, col_agg, layout):
    A = CASES[name]()
    with host(bd, A, col_agg=col_agg, record_layout=layout == "records") as M:
        assert M.stats()["lane_layout"] == (layout == "lanes")
        assert_same_structure(bd, A, M, col_agg=col_agg)
        assert_roundtrip(M, A)


@pytest.mark.parametrize("th1,th2", [(0, 0), (16, 64), (32, 128), (257 - 1, 256), (1, 255)])
def test_thresholds(bd, th1, th2):
    A = I.random_csr(96, 96, 0.35, 9)
    with host(bd, A, th1=th1, th2=th2, col_agg=0) as M:
        assert_same_structure(bd, A, M, col_agg=0, th1=th1, th2=th2)
        assert_roundtrip(M, A)


def test_explicit_zeros_survive_dense_tiles(bd):
    # a full 16x16 tile (Dense) with some stored values equal to +0.0 and -0.0
    idx = np.arange(256)
    v = I.uniform_pm1(1, 2, 256)
    v[[3, 77, 200]] = 0.0
    v[[5]] = -0.0
    A = I.csr_from_coo(16, 16, idx // 16, idx % 16, v, sum_duplicates=False)
    # drop two entries so that the tile has absent positions too
    keep = np.ones(256, bool); keep[[10, 11]] = False
    A = I.csr_from_coo(16, 16, (idx // 16)[keep], (idx % 16)[keep], v[keep], sum_duplicates=False)
    for rec in (False, True):
        with host(bd, A, record_layout=rec) as M:
            assert M.stats()["n_fmt"][B.FMT_DENSE] == 1
            assert_roundtrip(M, A)


def test_worked_example(bd):
    from test_oracle_blocked import example_32x48
    A = example_32x48()
    with host(bd, A) as M:
        g = M.export_blocked()
        assert g["aggregated"]
        assert g["type"].tolist() == [B.FMT_COO, B.FMT_DENSE, B.FMT_COO]
        st = M.stats()
    with host(bd, A, col_agg=0) as M0:
        st0 = M0.stats()
        assert st0["model_bytes_cb"] == 2463 and st0["model_bytes_csr"] == 3276
        assert st0["model_bytes_bsr16"] == 10272


def test_units_and_load_balance_invariants(bd):
    A = I.rmat(12, 16, seed=9)
    with host(bd, A) as M:
        st = M.stats()
        assert st["n_units"] >= 1 and st["n_workers"] == 1
        # host-only handles plan for one worker: every unit goes to it
        assert st["worker_load_max"] == pytest.approx(st["worker_load_mean"])
        assert st["mults_per_run"] >= A.nnz


def test_empty_and_degenerate(bd):
    for m, n in ((0, 0), (5, 0), (0, 7), (17, 33)):
        A = I.CSR(m, n, np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
        with host(bd, A) as M:
            st = M.stats()
            assert st["n_tiles"] == 0 and st["nnz"] == 0
            assert_roundtrip(M, A)


@pytest.mark.parametrize("bad", ["unsorted", "duplicate", "col_range", "rowptr", "neg_col"])
def test_rejects_non_canonical(bd, bad):
    A = I.random_csr(40, 40, 0.3, 3)
    col = A.col.copy(); rp = A.row_ptr.copy()
    if bad == "unsorted":
        r = np.flatnonzero(np.diff(rp) >= 2)[0]; k = rp[r]
        col[k], col[k + 1] = col[k + 1], col[k]
    elif bad == "duplicate":
        r = np.flatnonzero(np.diff(rp) >= 2)[0]; k = rp[r]
        col[k + 1] = col[k]
    elif bad == "col_range":
        col[-1] = 40
    elif bad == "neg_col":
        col[0] = -1
    elif bad == "rowptr":
        rp[5] = rp[6] + 1
    B_ = I.CSR(A.m, A.n, rp, col, A.val)
    with pytest.raises(bd.CbspmvError) as e:
        host(bd, B_)
    assert e.value.status == 2
    assert "row" in str(e.value) or "column" in str(e.value)


def test_rejects_bad_options(bd):
    A = I.random_csr(20, 20, 0.3, 3)
    for kw in ({"th1": 40, "th2": 30}, {"th2": 300}, {"col_agg": 2}, {"unit_work": -1}, {"device": -5}):
        with pytest.raises(bd.CbspmvError) as e:
            host(bd, A, **{k: v for k, v in kw.items() if k != "device"}) if "device" not in kw else \
                bd.BlockedMatrix(A, device=kw["device"])
        assert e.value.status == 1
    # an unknown value type is rejected (the four types of cbspmv_dtype_t are accepted)
    csr, _keep, _ = bd._csr_struct(A)
    o = bd._make_opts(device=-1)
    o.value_dtype = 9
    h = ctypes.c_void_p(None)
    assert bd.lib().cbspmv_analyze(ctypes.byref(csr), ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert h.value is None


def test_null_and_invalid_handles(bd):
    L = bd.lib()
    assert L.cbspmv_destroy(None) == 0
    assert L.cbspmv_run(None, None, None, 1.0, 0.0, None) == 1
    assert b"invalid handle" in L.cbspmv_last_error()
    s = bd.Stats()
    assert L.cbspmv_get_stats(None, ctypes.byref(s)) == 1
    A = I.random_csr(20, 20, 0.3, 3)
    with host(bd, A) as M:
        assert L.cbspmv_run(M.handle, None, None, 1.0, 0.0, None) == 1     # host-only handle
        assert b"host-only" in L.cbspmv_last_error()


def test_storage_model_matches_oracle_formula(bd):
    A = I.random_csr(300, 280, 0.02, 44)
    with host(bd, A, col_agg=0, th1=257 - 1, th2=256) as M:   # every tile COO
        st = M.stats()
        S = B.blocked_structure(A, col_agg=0, th1=256, th2=256)
        ref = B.storage_bytes(A.m, A.nnz, S.tile_nnz.size, (A.m + 15) // 16)
        assert st["model_bytes_cb"] == ref["cb_coo"]
        assert st["model_bytes_csr"] == ref["csr"]
        assert st["model_bytes_bsr16"] == ref["bsr16"]
        assert st["n_fmt"][0] == S.tile_nnz.size


def test_schedule_mode_follows_piece_sizes(bd):
    """Units whose rows hold one or two entries per tile get single-entry schedules; the
    FEM matrix's 3x3 blocks (pieces of about three entries) keep 3-entry chunks."""
    with host(bd, I.rmat(13, 16, seed=2), record_layout=True) as M:
        st = M.stats()
        assert st["n_entry_mode_units"] > 0.15 * st["n_units"]
    with host(bd, I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3),
              record_layout=True) as M:
        st = M.stats()
        assert st["n_entry_mode_units"] < 0.1 * st["n_units"]
        # 3x3 blocks: the chunks of (nearly) every unit cover consecutive columns
        assert st["n_xseq_units"] > 0.8 * st["n_units"]
        assert_roundtrip(M, I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3))


def test_value_map_option_keeps_the_structure(bd):
    A = I.random_csr(203, 157, 0.07, 5)
    with host(bd, A) as M0, host(bd, A, keep_value_map=True) as M1:
        a, b = M0.export_blocked(), M1.export_blocked()
        for key in ("blk_row", "blk_col", "nnz", "type", "cols_offset", "restore_cols"):
            assert np.array_equal(a[key], b[key])
        assert_roundtrip(M1, A)
        # a host-only handle cannot re-pack on a device
        with pytest.raises(bd.CbspmvError):
            M1.update_values(A.val)


def test_fma_slot_count(bd):
    """Record layout: fma_slots counts whole lanes (32 per chunk row) and at least one slot
    per entry; two hand-counted cases: a 16x16 diagonal is one unit of 16 single-entry chunks
    (rounded up to 2 descriptor rows of 32 lanes, 1 slot each); a dense 16x16 block is 16
    rows of six consecutive-column chunks (96 chunks: 4 descriptor rows of 32 lanes, 3 slots
    each)."""
    for A in (I.rmat(12, 16, seed=4), I.laplacian2d(64), I.random_csr(333, 517, 0.2, 11),
              I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)):
        with host(bd, A, record_layout=True) as M:
            st = M.stats()
        assert st["fma_slots"] % 32 == 0 and st["fma_slots"] >= A.nnz
    r = np.arange(16)
    with host(bd, I.csr_from_coo(16, 16, r, r, np.ones(16)), record_layout=True) as M:
        st = M.stats()
    assert st["n_entry_mode_units"] == 1 and st["fma_slots"] == 64
    r, c = np.repeat(np.arange(16), 16), np.tile(np.arange(16), 16)
    with host(bd, I.csr_from_coo(16, 16, r, c, np.ones(256)), record_layout=True) as M:
        st = M.stats()
    assert st["n_xseq_units"] == 1 and st["fma_slots"] == 384


def test_lane_layout_fma_slots_and_units(bd):
    """Lane-stream layout: every unit issues 32 x ceil(entries / 32) FMA slots (no Dense
    zero fill, no chunk rounding). Hand-counted: a 16x16 diagonal is one unit of 16
    entries (one step: 32 slots); a full 16x16 block is one Dense sub-block of 256 entries
    (8 steps: 256 slots, every slot useful); a FEM block row of the 3x3 band (16 rows x 81
    entries = 1,296) fits one unit of 41 steps."""
    r = np.arange(16)
    with host(bd, I.csr_from_coo(16, 16, r, r, np.ones(16))) as M:
        st = M.stats()
    assert st["lane_layout"] == 1 and st["n_units"] == 1 and st["fma_slots"] == 32
    r, c = np.repeat(np.arange(16), 16), np.tile(np.arange(16), 16)
    with host(bd, I.csr_from_coo(16, 16, r, c, np.ones(256))) as M:
        st = M.stats()
    assert st["n_fmt"][B.FMT_DENSE] == 1 and st["fma_slots"] == 256
    F = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    with host(bd, F) as M:
        st = M.stats()
        assert_roundtrip(M, F)
    # whole block rows of the band hold 1,296 entries: well over 97% of the slots are useful
    assert st["n_split_units"] == 0
    assert F.nnz / st["fma_slots"] > 0.97
    for A in (I.rmat(12, 16, seed=4), I.laplacian2d(64), I.random_csr(333, 517, 0.2, 11)):
        with host(bd, A) as M:
            st = M.stats()
            assert_roundtrip(M, A)
        assert st["fma_slots"] % 32 == 0 and A.nnz <= st["fma_slots"] < A.nnz + 32 * st["n_units"]


def test_lane_layout_cuts_long_block_rows(bd):
    """A block row with more sub-blocks than one unit's x slots (32) is cut into parts whose
    partial sums the combine adds; the parts keep every entry once (round trip)."""
    A = I.isolated_entries_block_row(tiles=70)
    with host(bd, A, col_agg=0) as M:
        st = M.stats()
        assert_roundtrip(M, A)
        blk = M.export_blocked()
    ntiles = len(blk["nnz"])
    assert ntiles > 32 and st["n_split_units"] >= (ntiles + 31) // 32 and st["n_split_rows"] == 1


def test_direct_descriptors_where_columns_are_known_per_chunk(bd):
    """Single-entry and consecutive-column units of at most 512 chunks carry direct (value
    offset, tile, column, entry) descriptors and keep their values in load order after
    the coordinate parts; export still returns every value bit-exactly (FP64) or as the
    oracle's rounding of it (BF16)."""
    from oracle import lowprec as L
    A = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    with host(bd, A, record_layout=True) as M:
        st = M.stats()
        assert_roundtrip(M, A)
    assert st["n_direct_units"] == st["n_xseq_units"] + st["n_entry_mode_units"] > 0
    with host(bd, A, value_dtype="bf16", record_layout=1) as M:
        st = M.stats()
        rp, col, val = M.export_csr()
    assert st["n_direct_units"] == st["n_xseq_units"] + st["n_entry_mode_units"] > 0
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    assert np.array_equal(val.view(np.uint64), L.round_to_format(A.val, "bf16").view(np.uint64))
    R = I.rmat(13, 16, seed=2)
    with host(bd, R, record_layout=True) as M:
        st = M.stats()
        assert_roundtrip(M, R)
    assert 0 < st["n_direct_units"] <= st["n_entry_mode_units"] + st["n_xseq_units"]
    r, c = np.repeat(np.arange(16), 16), np.tile(np.arange(16), 16)
    D = I.csr_from_coo(16, 16, r, c, I.normal(4, I.TAG_VAL, 256))
    with host(bd, D, record_layout=True) as M:      # one Dense tile
        assert M.stats()["n_direct_units"] == 1 and M.stats()["n_fmt"][2] == 1
        assert_roundtrip(M, D)


def test_long_single_entry_unit_keeps_16bit_descriptors(bd):
    """540 single-entry chunks in one unit (27 per tile, pieces of 1.7 entries): more than
    direct descriptors cover, so the unit keeps 16-bit descriptors."""
    A = I.isolated_entries_block_row()
    with host(bd, A, col_agg=0, record_layout=True) as M:
        st = M.stats()
        assert_roundtrip(M, A)
    assert st["n_units"] == 1 and st["n_entry_mode_units"] == 1 and st["n_direct_units"] == 0
    assert st["fma_slots"] == 32 * 18       # 540 chunks: 17 per lane, 18 descriptor rows


def test_analysis_does_not_depend_on_the_thread_count(bd, tmp_path):
    """The same analysis with one host thread, eight and all of them (CBSPMV_HOST_THREADS,
    each in a child process): equal statistics (apart from the time) and byte-equal
    exports. The inputs are large enough that every chunked loop of the analysis (block
    rows, units, schedules, the in-place re-layout) runs as many chunks."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = """
import hashlib, json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2605_18515_gb300 import build, inputs as I
build.build()
from paper_2605_18515_gb300 import binding as bd
out = {}
for name, A in (("fem", I.fem_block_band(n_rows=60000, n_block_rows=20000, half_band=800, seed=3)),
                ("rmat", I.rmat(15, 16, seed=4))):
    for dt in ("f64", "bf16"):
        with bd.BlockedMatrix(A, device=-1, keep_value_map=True, value_dtype=dt) as M:
            st = M.stats(); st.pop("analyze_ms")
            rp, col, val = M.export_csr()
            blk = M.export_blocked()
        h = hashlib.sha256()
        for arr in (rp, col, val, *[np.asarray(blk[k]) for k in sorted(blk)]):
            h.update(np.ascontiguousarray(arr).tobytes())
        out[name + "_" + dt] = {"stats": st, "digest": h.hexdigest(), "nnz": int(col.size)}
print(json.dumps(out))
""".replace("ROOT", repr(root))
    res = {}
    for threads in ("1", "8", None):
        env = dict(os.environ)
        env.pop("CBSPMV_HOST_THREADS", None)
        if threads:
            env["CBSPMV_HOST_THREADS"] = threads
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        assert p.returncode == 0, p.stderr[-2000:]
        res[threads] = json.loads(p.stdout.strip().splitlines()[-1])
    assert res["1"]["fem_f64"]["stats"]["n_block_rows"] > 3000
    assert res["1"]["rmat_f64"]["stats"]["n_units"] > 1000
    assert res["1"] == res["8"] == res[None]


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", ["random_ragged", "random_dense", "laplace2d_64", "rmat10"])
@pytest.mark.parametrize("col_agg", [0, 1])
def test_reduced_type_lane_layout_roundtrip(bd, fmt, name, col_agg):
    """record_layout 2: the lane-stream layout for the 4- and 2-byte value types (steps in
    groups of 8, plain sub-blocks with one gather entry each). The blocked structure is the
    oracle's; export returns every value as the oracle's rounding of it to the storage type."""
    from oracle import lowprec as L
    A = CASES[name]() if name in CASES else I.rmat(10, 16, seed=3)
    with host(bd, A, value_dtype=fmt, record_layout=2, col_agg=col_agg) as M:
        st = M.stats()
        assert st["lane_layout"] == 1
        assert_same_structure(bd, A, M, col_agg=col_agg)
        rp, col, val = M.export_csr()
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    assert np.array_equal(val, L.round_to_format(A.val, fmt))
    # values: one slot per lane and step (no padding of the last group to 8 steps), 32 lanes;
    # words 2 bytes per slot, each unit's rounded up to 4 steps
    vs = {"f32": 4, "bf16": 2, "f16": 2}[fmt]
    assert st["fma_slots"] % 32 == 0 and A.nnz <= st["fma_slots"] < A.nnz + 32 * st["n_units"]
    words = st["stream_bytes"] - st["fma_slots"] * vs
    assert 2 * st["fma_slots"] <= words <= 2 * st["fma_slots"] + 3 * 64 * st["n_units"] and words % 256 == 0


def test_plain_gather_lists_hold_one_column_per_sub_block(bd):
    """Reduced-type lane units without aggregation keep the first column of each plain
    sub-block in their gather list (padded to 4 entries); with aggregation, and in the FP64
    lane layout, 16 columns per sub-block."""
    from oracle import lowprec as L
    A = I.random_csr(300, 280, 0.1, 4)
    with host(bd, A, col_agg=0, value_dtype="bf16", record_layout=2) as M0, \
            host(bd, A, col_agg=1, value_dtype="bf16", record_layout=2) as M1, host(bd, A, col_agg=0) as M2:
        s0, s1, s2 = M0.stats(), M1.stats(), M2.stats()
        for M in (M0, M1):
            rp, col, val = M.export_csr()
            assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
            assert np.array_equal(val, L.round_to_format(A.val, "bf16"))
        assert_roundtrip(M2, A)
    g2 = s2["metadata_bytes"] - s2["n_tiles"] * 16 - 32 * s2["n_units"]
    assert g2 == 4 * 16 * s2["n_tiles"]
    tile_bytes = 16  # one CbTile record per sub-block
    g0 = s0["metadata_bytes"] - s0["n_tiles"] * tile_bytes - 32 * s0["n_units"]
    g1 = s1["metadata_bytes"] - s1["n_tiles"] * tile_bytes - 32 * s1["n_units"]
    assert g1 == 4 * 16 * s1["n_tiles"]
    assert s0["n_tiles"] * 4 <= g0 < (s0["n_tiles"] + 3 * s0["n_units"]) * 4 + 1


@pytest.mark.parametrize("fmt", ["f64", "bf16"])
def test_uint16_gather_lists(bd, fmt):
    """Per-slot gather lists become uint16 offsets from the unit's first column when the
    unit's columns span fewer than 65,535 values (a FEM band with aggregation: every unit),
    and stay 32-bit when they do not (a matrix whose rows each reach both ends of 200,000
    columns). Both decode back to the input CSR bit for bit; the gather bytes count 2 or 4
    per slot."""
    from oracle import lowprec as L
    fem = I.fem_block_band(n_rows=6000, n_block_rows=2000, half_band=300, seed=3)
    # 64 rows, each with entries at columns 0..7 and 199,990..199,999
    rr = np.repeat(np.arange(64), 16)
    cc = np.tile(np.r_[np.arange(8), 199_990 + np.arange(10)[:8]], 64)
    wide = I.csr_from_coo(64, 200_000, rr, cc, I.uniform_pm1(5, 1, rr.size))
    lay = {} if fmt == "f64" else {"record_layout": 2}
    for A, agg, want in ((fem, 1, "all"), (wide, 0, "none"), (wide, 1, "none")):
        with host(bd, A, value_dtype=fmt, col_agg=agg, **lay) as M:
            st = M.stats()
            assert st["lane_layout"] == 1
            if want == "all":
                assert st["n_g16_units"] == st["n_units"] > 0
                assert st["gather_list_bytes"] == 2 * 16 * st["n_tiles"]
            elif fmt != "f64" and agg == 0:   # plain sub-blocks: one 32-bit entry each
                assert st["n_g16_units"] == 0
                assert st["gather_list_bytes"] == 4 * ((st["n_tiles"] + 3) // 4 * 4) and st["n_units"] == 1
            else:
                assert st["n_g16_units"] == 0
                assert st["gather_list_bytes"] == 4 * 16 * st["n_tiles"]
            rp, col, val = M.export_csr()
        assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
        if fmt == "f64":
            assert np.array_equal(val.view(np.uint64), A.val.view(np.uint64))
        else:
            assert np.array_equal(val, L.round_to_format(A.val, fmt))
