// Host analysis of a CSR matrix into the blocked layout (Sec. 3 of the paper):
//   1. validation of the canonical CSR input;
//   2. 16x16 tiling of each block row and the super-sparse share that decides column
//      aggregation (Sec. 3.3.1, threshold th0);
//   3. per block row: column aggregation (restore_cols / cols_offset), re-tiling, per-tile
//      format selection (Sec. 3.3.2, th1 / th2) and packing of every tile into one
//      16-byte aligned record behind its virtual pointer (Sec. 3.2);
//   4. cutting the tile sequence into units of work for the kernel's warps and the
//      load balance of units over the persistent thread blocks (Sec. 3.4): units sorted
//      by cost, each handed to the least-loaded thread block taken from a min-heap.
// Block rows are independent, so steps 2-3 run on all host cores.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>

#include "cb_plan.h"
#include "cb_round.h"

namespace cb {
namespace {

// Analysis threads: the host's hardware threads (at most 64), or CBSPMV_HOST_THREADS
// (1..64) when set. The result does not depend on the count.
int host_threads() {
  if (const char* env = std::getenv("CBSPMV_HOST_THREADS")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v >= 1 && v <= 64) return (int)v;
  }
  unsigned h = std::thread::hardware_concurrency();
  if (h == 0) h = 1;
  return (int)std::min(h, 64u);
}

// Runs f(lo, hi) over [0, n) in chunks on all host cores.
void parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& f) {
  int T = host_threads();
  if (n <= grain || T == 1) {
    f(0, n);
    return;
  }
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      int64_t lo = next.fetch_add(grain);
      if (lo >= n) break;
      f(lo, std::min(n, lo + grain));
    }
  };
  std::vector<std::thread> th;
  int nt = (int)std::min<int64_t>(T, (n + grain - 1) / grain);
  for (int i = 1; i < nt; ++i) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
}

inline int select_format(int nnz, int th1, int th2) {
  if (nnz < th1) return CB_FMT_COO;
  if (nnz > th2) return CB_FMT_DENSE;
  return CB_FMT_CSR;
}

inline uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

// Bytes of one packed tile record.
inline uint32_t record_bytes(int fmt, int nnz, int vsize) {
  switch (fmt) {
    case CB_FMT_COO: return align16(align16((uint32_t)nnz) + (uint32_t)nnz * vsize);
    case CB_FMT_CSR: return align16(align16(17u + (uint32_t)nnz) + (uint32_t)nnz * vsize);
    default: return align16(32u + 256u * vsize);
  }
}

struct BlockRowOut {
  std::vector<uint8_t> bytes;      // packed records of this block row
  std::vector<uint32_t> off;       // record offsets inside `bytes`
  std::vector<int32_t> bcol;       // block column per tile
  std::vector<uint16_t> nnz;
  std::vector<uint8_t> fmt;
  std::vector<uint8_t> rowcnt;     // 16 per tile: multiply-adds of each tile row
  std::vector<int32_t> distinct;   // distinct columns in order (aggregated only)
  std::vector<std::pair<int64_t, uint32_t>> vslot;   // (CSR position, value byte offset in `bytes`)
};

// Sorts v, made of nruns consecutive ascending runs (run i = [bounds[i], bounds[i + 1])),
// by merging the runs pairwise; tmp is scratch. Same result as std::sort for unique keys.
template <class T>
void merge_sorted_runs(std::vector<T>& v, std::vector<T>& tmp, const size_t* bounds, int nruns) {
  tmp.resize(v.size());
  for (int w = 1; w < nruns; w *= 2) {
    for (int i = 0; i < nruns; i += 2 * w) {
      const size_t lo = bounds[i], mid = bounds[std::min(i + w, nruns)], hi = bounds[std::min(i + 2 * w, nruns)];
      std::merge(v.begin() + lo, v.begin() + mid, v.begin() + mid, v.begin() + hi, tmp.begin() + lo);
    }
    v.swap(tmp);
  }
}

// Entries of one block row as (key = col << 4 | local row, CSR position), sorted by key.
// Each row's columns ascend (canonical CSR), so the rows are sorted runs to be merged.
void gather_block_row(const cbspmv_csr_t& A, int64_t b, std::vector<std::pair<uint64_t, int64_t>>& e,
                      std::vector<std::pair<uint64_t, int64_t>>& tmp) {
  e.clear();
  int64_t r0 = b * CB_BLK, r1 = std::min<int64_t>(A.m, r0 + CB_BLK);
  size_t bounds[CB_BLK + 1];
  int nr = 0;
  bounds[0] = 0;
  for (int64_t r = r0; r < r1; ++r) {
    for (int64_t k = A.row_ptr[r]; k < A.row_ptr[r + 1]; ++k)
      e.emplace_back(((uint64_t)(uint32_t)A.col_idx[k] << 4) | (uint64_t)(r - r0), k);
    bounds[++nr] = e.size();
  }
  merge_sorted_runs(e, tmp, bounds, nr);
}

}  // namespace

static_assert(CB_B_MAX <= 8192 && CB_B_MAX_4 <= 8192 && CB_B_MAX_2 <= 8192,
              "direct chunk descriptors hold value offsets / 2 in 12 bits within a unit's stream bytes");

// Column (0..15, in the tile) of entry e of tile tg, from its packed record (row-major
// entry order; Dense entry e is row e / 16, column e % 16).
static inline uint32_t entry_col(const Plan& p, size_t tg, uint32_t e) {
  const CbTile& t = p.tiles[tg];
  if (t.fmt == CB_FMT_DENSE) return e & 15u;
  const uint8_t* rec = p.stream.data() + (size_t)t.vp16 * 16;
  const uint8_t* idx = rec + (t.fmt == CB_FMT_CSR ? 17 : 0);
  return idx[e] >> 4;
}

// Entries of the chunk starting at entry e (at most len) whose columns are consecutive.
static inline uint32_t xseq_run(const Plan& p, size_t tg, uint32_t e, uint32_t len) {
  uint32_t k = 1;
  const uint32_t c0 = entry_col(p, tg, e);
  while (k < len && entry_col(p, tg, e + k) == c0 + k) ++k;
  return k;
}

// Chunks of the piece (tile tg, row rr, entries s0 .. s0 + c - 1) when chunks of up to
// CB_CHUNK entries also stop at column gaps.
static inline uint64_t xseq_chunks(const Plan& p, size_t tg, int rr, uint32_t s0, uint32_t c) {
  (void)rr;
  uint64_t n = 0;
  for (uint32_t o = 0; o < c;) {
    o += xseq_run(p, tg, s0 + o, std::min<uint32_t>(CB_CHUNK, c - o));
    ++n;
  }
  return n;
}

namespace {

// Stores v in the handle's value type, rounded to nearest (ties to even) directly from
// the FP64 input; the rounded value is exact in the stored type.
void write_value(uint8_t* dst, double v, int dtype) {
  const uint64_t bits = storage_bits(v, dtype);
  std::memcpy(dst, &bits, dtype == CBSPMV_F64 ? 8 : dtype == CBSPMV_F32 ? 4 : 2);   // little endian
}

// The stored value at src widened exactly to double.
double read_value(const uint8_t* src, int dtype) {
  switch (dtype) {
    case CBSPMV_F64: { double d; std::memcpy(&d, src, 8); return d; }
    case CBSPMV_F32: { float f; std::memcpy(&f, src, 4); return f; }
    case CBSPMV_BF16: {
      uint16_t h; std::memcpy(&h, src, 2);
      const uint32_t b = (uint32_t)h << 16;
      float f; std::memcpy(&f, &b, 4);
      return f;
    }
    default: {
      uint16_t h; std::memcpy(&h, src, 2);
      const double sign = (h & 0x8000u) ? -1.0 : 1.0;
      const int ex = (h >> 10) & 31, fr = h & 1023;
      if (ex == 31) return fr ? NAN : sign * INFINITY;
      if (ex == 0) return sign * std::ldexp((double)fr, -24);
      return sign * std::ldexp((double)(1024 + fr), ex - 25);
    }
  }
}

int value_size(int dtype) { return dtype == CBSPMV_F64 ? 8 : dtype == CBSPMV_F32 ? 4 : 2; }

void build_block_row(const cbspmv_csr_t& A, int64_t b, bool agg, int th1, int th2, int dtype, bool keep_slots,
                     std::vector<std::pair<uint64_t, int64_t>>& e, std::vector<std::pair<uint64_t, int64_t>>& tmp,
                     BlockRowOut& out) {
  const int vsize = value_size(dtype);
  gather_block_row(A, b, e, tmp);
  out = BlockRowOut();
  const size_t ne = e.size();
  if (ne == 0) return;
  // aggregated column of every entry (Sec. 3.3.1): rank of its column among the block
  // row's distinct columns; plain: the column itself.
  std::vector<uint32_t> acol(ne);
  if (agg) {
    int64_t prev = -1;
    uint32_t rank = 0;
    for (size_t i = 0; i < ne; ++i) {
      int64_t c = (int64_t)(e[i].first >> 4);
      if (c != prev) {
        if (prev >= 0) ++rank;
        out.distinct.push_back((int32_t)c);
        prev = c;
      }
      acol[i] = rank;
    }
  } else {
    for (size_t i = 0; i < ne; ++i) acol[i] = (uint32_t)(e[i].first >> 4);
  }
  std::vector<std::pair<uint32_t, int64_t>> tile;  // (row * 16 + col in tile, CSR position)
  size_t a = 0;
  while (a < ne) {
    uint32_t bj = acol[a] >> 4;
    size_t z = a;
    while (z < ne && (acol[z] >> 4) == bj) ++z;
    // row-major order inside the tile: the entries come by (column, row), so a stable
    // counting sort by row leaves each row's columns ascending
    uint32_t start[17] = {0};
    for (size_t k = a; k < z; ++k) start[(e[k].first & 15u) + 1]++;
    for (int r = 0; r < 16; ++r) start[r + 1] += start[r];
    tile.resize(z - a);
    for (size_t k = a; k < z; ++k) {
      const uint32_t lr = (uint32_t)(e[k].first & 15u), lc = acol[k] & 15u;
      tile[start[lr]++] = {lr * 16u + lc, e[k].second};
    }
    int nnz = (int)tile.size();
    int fmt = select_format(nnz, th1, th2);
    {
      size_t rc0 = out.rowcnt.size();
      out.rowcnt.resize(rc0 + 16, 0);
      for (auto& t : tile) out.rowcnt[rc0 + (t.first >> 4)]++;
      if (fmt == CB_FMT_DENSE)
        for (int r = 0; r < 16; ++r) out.rowcnt[rc0 + r] = 16;   // zero fill is multiplied too
    }
    uint32_t rb = record_bytes(fmt, nnz, vsize);
    uint32_t base = (uint32_t)out.bytes.size();
    out.bytes.resize(base + rb, 0);
    uint8_t* rec = out.bytes.data() + base;
    if (fmt == CB_FMT_DENSE) {
      for (auto& t : tile) {
        uint32_t pos = t.first;  // row * 16 + col
        rec[pos >> 3] |= (uint8_t)(1u << (pos & 7));
        write_value(rec + 32 + pos * vsize, A.val[t.second], dtype);
        if (keep_slots) out.vslot.emplace_back(t.second, base + 32 + pos * vsize);
      }
    } else {
      uint8_t* idx = rec;
      if (fmt == CB_FMT_CSR) {
        // 17 row-pointer bytes
        int cnt[16] = {0};
        for (auto& t : tile) cnt[t.first >> 4]++;
        rec[0] = 0;
        for (int r = 0; r < 16; ++r) rec[r + 1] = (uint8_t)(rec[r] + cnt[r]);
        idx = rec + 17;
      }
      uint32_t voff = align16((uint32_t)(idx - rec) + (uint32_t)nnz);
      for (int i = 0; i < nnz; ++i) {
        uint32_t lr = tile[i].first >> 4, lc = tile[i].first & 15u;
        idx[i] = (uint8_t)(lr | (lc << 4));          // row low nibble, col high nibble
        write_value(rec + voff + (uint32_t)i * vsize, A.val[tile[i].second], dtype);
        if (keep_slots) out.vslot.emplace_back(tile[i].second, base + voff + (uint32_t)i * vsize);
      }
    }
    out.off.push_back(base);
    out.bcol.push_back((int32_t)bj);
    out.nnz.push_back((uint16_t)nnz);
    out.fmt.push_back((uint8_t)fmt);
    a = z;
  }
}

}  // namespace

void host_parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& f) {
  parallel_for(n, grain, f);
}
int tile_format(int nnz, int th1, int th2) { return select_format(nnz, th1, th2); }

// Sizes and array pointers of a CSR (the contents are checked by validate on the host and
// by the device analysis on the GPU).
cbspmv_status_t validate_shape(const cbspmv_csr_t& A, std::string* msg) {
  if (A.m < 0 || A.n < 0 || A.nnz < 0 || A.m >= (1LL << 31) || A.n >= (1LL << 31) ||
      A.nnz >= (1LL << 31)) {
    *msg = "matrix dimensions out of range";
    return CBSPMV_ERR_INVALID;
  }
  if (!A.row_ptr || (A.nnz > 0 && (!A.col_idx || !A.val))) {
    *msg = "NULL CSR array";
    return CBSPMV_ERR_INVALID;
  }
  return CBSPMV_OK;
}

namespace {

cbspmv_status_t validate(const cbspmv_csr_t& A, std::string* msg) {
  const cbspmv_status_t st0 = validate_shape(A, msg);
  if (st0 != CBSPMV_OK) return st0;
  if (A.row_ptr[0] != 0 || A.row_ptr[A.m] != A.nnz) {
    *msg = "row_ptr must start at 0 and end at nnz";
    return CBSPMV_ERR_NOT_CANONICAL;
  }
  std::atomic<int> bad(0);
  parallel_for(A.m, 1 << 14, [&](int64_t lo, int64_t hi) {
    for (int64_t r = lo; r < hi && !bad.load(std::memory_order_relaxed); ++r) {
      int64_t a = A.row_ptr[r], z = A.row_ptr[r + 1];
      if (z < a || a < 0 || z > A.nnz) { bad = 1; return; }
      int64_t prev = -1;
      for (int64_t k = a; k < z; ++k) {
        int64_t c = A.col_idx[k];
        if (c <= prev || c >= A.n) { bad = 2; return; }
        prev = c;
      }
    }
  });
  if (bad.load() == 1) { *msg = "row_ptr is not non-decreasing"; return CBSPMV_ERR_NOT_CANONICAL; }
  if (bad.load() == 2) {
    *msg = "column indices must be strictly increasing within a row and lie in [0, n)";
    return CBSPMV_ERR_NOT_CANONICAL;
  }
  return CBSPMV_OK;
}

}  // namespace

// Lane-stream programs of every unit (layout in cb_layout.h), built from the packed records
// after the load balance (so each worker's units are contiguous in the arrays). rowcnt:
// entries of each (tile, row) of the records (16 per row for Dense tiles, whose present
// entries come from the presence bitmap). Also composes the value map with the move of
// every value from its record to its lane position, and counts the FMA slots.
// Offsets of every unit's values, entry words and gather list in the lane-stream arrays
// (units in worker order), and the unit descriptors without their flags. The sizes of the
// three arrays go to p.n_lane_vals, p.n_lane_words and p.n_lane_gcols; p.fma_slots is the
// value count.
cbspmv_status_t lane_offsets(Plan& p, std::vector<uint64_t>* voff_out, std::vector<uint64_t>* woff_out,
                             std::vector<uint64_t>* goff_out, std::string* msg) {
  const size_t nun = p.units.size();
  std::vector<uint64_t>& voff = *voff_out;
  std::vector<uint64_t>& woff = *woff_out;
  std::vector<uint64_t>& goff = *goff_out;
  voff.assign(nun + 1, 0);
  woff.assign(nun + 1, 0);
  goff.assign(nun + 1, 0);
  const bool grouped = p.vsize != 8;    // the reduced-type layout: full groups of 8 steps
  // one gather-list entry per plain sub-block (4- and 2-byte value types; the FP64 kernel
  // keeps one entry per x slot, which measured faster there)
  const bool plainx = !p.aggregated && grouped;
  std::vector<uint64_t> steps(nun);
  for (size_t i = 0; i < nun; ++i) {
    const CbUnit& u = p.units[i];
    uint64_t W = 0;
    for (uint32_t t = 0; t < u.ntiles; ++t) W += p.tiles[u.tile_lo + t].nnz;
    const uint64_t S = (W + CB_VLANES - 1) / CB_VLANES;
    steps[i] = S;
    voff[i + 1] = voff[i] + S;
    woff[i + 1] = woff[i] + (S + 3) / 4;
    goff[i + 1] = goff[i] + (plainx ? (u.ntiles + 3ull) / 4 * 4 : 16ull * u.ntiles);
  }
  if (voff[nun] >= (1ull << 32) || woff[nun] >= (1ull << 32) || goff[nun] >= (1ull << 32)) {
    *msg = "lane stream too large";
    return CBSPMV_ERR_UNSUPPORTED;
  }
  try {
    p.lane_units.resize(nun);
  } catch (...) {
    *msg = "host allocation failed";
    return CBSPMV_ERR_OOM;
  }
  for (size_t i = 0; i < nun; ++i) {
    const CbUnit& u = p.units[i];
    CbLaneUnit& L = p.lane_units[i];
    L = CbLaneUnit{};
    L.vals = (uint32_t)voff[i];
    L.words = (uint32_t)woff[i];
    L.gcols = (uint32_t)goff[i];
    L.brow_lo = u.brow_lo;
    L.steps = (uint16_t)steps[i];
    L.nslots = (uint16_t)(16 * u.ntiles);
    L.nrows = (uint16_t)std::min<int64_t>((int64_t)CB_BLK * u.nbr, p.m - (int64_t)u.brow_lo * CB_BLK);
    L.flags = plainx ? CB_LUNIT_PLAINX : 0;
    L.slot = u.split >= 0 ? u.slot : 0xffffffffu;
  }
  p.n_lane_vals = (size_t)voff[nun] * CB_VLANES;
  p.n_lane_words = (size_t)woff[nun] * CB_VLANES;
  p.n_lane_gcols = (size_t)goff[nun];
  p.fma_slots = (int64_t)voff[nun] * CB_VLANES;
  return CBSPMV_OK;
}

// A unit's per-slot gather list g (u.nslots columns, -1 for none) rewritten in place as
// uint16 offsets from its smallest column when its columns span fewer than 65,535 values
// (CB_LUNIT_G16; 0xffff for none): the list's bytes halve for banded matrices. The words
// after the uint16 list keep their old contents (the list's space is not reclaimed).
static void compact_gather_list(CbLaneUnit& u, int32_t* g) {
  int64_t lo = INT64_MAX, hi = -1;
  for (uint32_t k = 0; k < u.nslots; ++k)
    if (g[k] >= 0) {
      lo = std::min<int64_t>(lo, g[k]);
      hi = std::max<int64_t>(hi, g[k]);
    }
  if (hi < 0 || hi - lo >= 0xffff) return;
  uint16_t h[CB_LANE_SLOTS];
  for (uint32_t k = 0; k < u.nslots; ++k) h[k] = g[k] < 0 ? (uint16_t)0xffffu : (uint16_t)(g[k] - lo);
  std::memcpy(g, h, 2u * u.nslots);
  u.flags |= CB_LUNIT_G16;
  u.gbase = (uint32_t)lo;
}

// Lane-stream programs of every unit (layout in cb_layout.h), built from the packed records
// after the load balance (so each worker's units are contiguous in the arrays). rowcnt:
// entries of each (tile, row) of the records (16 per row for Dense tiles, whose present
// entries come from the presence bitmap). Also composes the value map with the move of
// every value from its record to its lane position, and counts the FMA slots.
static cbspmv_status_t build_lane_programs(const cbspmv_csr_t& A, Plan& p, const std::vector<uint8_t>& rowcnt,
                                           std::string* msg) {
  const size_t nun = p.units.size();
  std::vector<uint64_t> voff, woff, goff;
  cbspmv_status_t st = lane_offsets(p, &voff, &woff, &goff, msg);
  if (st != CBSPMV_OK) return st;
  try {
    p.lane_vals.resize(p.n_lane_vals * (size_t)p.vsize);
    p.lane_words.resize(p.n_lane_words);
    p.lane_gcols.resize(p.n_lane_gcols);
  } catch (...) {
    *msg = "host allocation failed";
    return CBSPMV_ERR_OOM;
  }
  const uint32_t vs = (uint32_t)p.vsize;
  const bool grouped = vs != 8;
  // value index in the record stream -> value index in the lane stream (value map only)
  std::vector<uint32_t> moved(p.value_slot.empty() ? 0 : p.stream.size() / vs, UINT32_MAX);
  parallel_for((int64_t)nun, 128, [&](int64_t lo, int64_t hi) {
    struct Ent { uint16_t word; uint32_t vidx; };   // entry word, value index in the record stream
    std::vector<Ent> ent;
    for (int64_t i = lo; i < hi; ++i) {
      const CbUnit& u = p.units[i];
      const int64_t R = std::min<int64_t>((int64_t)CB_BLK * u.nbr, A.m - (int64_t)u.brow_lo * CB_BLK);
      ent.clear();
      // entries row by row: block row of the unit, row nibble, tile, column
      uint32_t t_begin = 0;
      for (int64_t brl = 0; brl < u.nbr; ++brl) {
        uint32_t t_end = t_begin;
        while (t_end < u.ntiles && (int64_t)p.tiles[u.tile_lo + t_end].brow - u.brow_lo == brl) ++t_end;
        for (int rr = 0; rr < 16; ++rr) {
          const int64_t row = brl * 16 + rr;
          if (row >= R) break;
          for (uint32_t t = t_begin; t < t_end; ++t) {
            const size_t tg = (size_t)(u.tile_lo + t);
            const CbTile& tr = p.tiles[tg];
            const size_t rec = (size_t)tr.vp16 * 16;
            if (tr.fmt == CB_FMT_DENSE) {
              const uint8_t* bm = p.stream.data() + rec;
              for (uint32_t c = 0; c < 16; ++c) {
                const uint32_t pos = 16u * rr + c;
                if (bm[pos >> 3] & (1u << (pos & 7)))
                  ent.push_back({(uint16_t)((16u * t + c) | ((uint32_t)row << 9)), (uint32_t)((rec + 32 + vs * pos) / vs)});
              }
            } else {
              const uint32_t c = rowcnt[tg * 16 + rr];
              if (!c) continue;
              uint32_t s0 = 0;
              for (int q = 0; q < rr; ++q) s0 += rowcnt[tg * 16 + q];
              const uint32_t ib = tr.fmt == CB_FMT_CSR ? 17u : 0u;
              const uint32_t va = align16(ib + tr.nnz);
              for (uint32_t e = s0; e < s0 + c; ++e) {
                const uint32_t col = p.stream[rec + ib + e] >> 4;
                ent.push_back({(uint16_t)((16u * t + col) | ((uint32_t)row << 9)), (uint32_t)((rec + va + vs * e) / vs)});
              }
            }
          }
        }
        t_begin = t_end;
      }
      const uint64_t W = ent.size();
      uint8_t* vals = p.lane_vals.data() + (size_t)voff[i] * CB_VLANES * vs;
      uint64_t* words = p.lane_words.data() + (size_t)woff[i] * CB_VLANES;
      std::fill(vals, vals + (size_t)(voff[i + 1] - voff[i]) * CB_VLANES * vs, (uint8_t)0);
      std::fill(words, words + (size_t)(woff[i + 1] - woff[i]) * CB_VLANES, ~0ull);
      int first_lane[CB_R_MAX], last_lane[CB_R_MAX];
      for (int r = 0; r < CB_R_MAX; ++r) first_lane[r] = last_lane[r] = -1;
      for (uint32_t l = 0; l < CB_VLANES; ++l) {
        const uint64_t c0 = (l * W) / CB_VLANES, c1 = ((l + 1) * W) / CB_VLANES;
        for (uint64_t k = c0; k < c1; ++k) {
          const uint64_t st = k - c0;
          const Ent& e = ent[k];
          const uint32_t S = p.lane_units[i].steps;
          const uint32_t vi = cb_lane_val_index(grouped, (uint32_t)st, l, S);
          std::memcpy(vals + (size_t)vi * vs, p.stream.data() + (size_t)e.vidx * vs, vs);
          uint64_t& w = words[cb_lane_word_index(grouped, (uint32_t)st, l, S)];
          const uint32_t sh = 16u * (uint32_t)(st % 4);
          w = (w & ~(0xffffull << sh)) | ((uint64_t)e.word << sh);
          if (!moved.empty()) moved[e.vidx] = (uint32_t)((size_t)voff[i] * CB_VLANES + vi);
          const int r = e.word >> 9;
          if (first_lane[r] < 0) first_lane[r] = (int)l;
          last_lane[r] = (int)l;
        }
      }
      int span_max = 0;
      for (int r = 0; r < CB_R_MAX; ++r)
        if (first_lane[r] >= 0) span_max = std::max(span_max, last_lane[r] - first_lane[r] + 1);
      // gather list: the first column of every plain sub-block, or the x column of every slot
      int32_t* g = p.lane_gcols.data() + goff[i];
      if (p.lane_units[i].flags & CB_LUNIT_PLAINX) {
        for (uint64_t k = 0; k < goff[i + 1] - goff[i]; ++k)
          g[k] = k < u.ntiles ? (int32_t)p.tiles[u.tile_lo + k].xbase : 0;
      }
      for (uint32_t t = 0; t < u.ntiles && !(p.lane_units[i].flags & CB_LUNIT_PLAINX); ++t) {
        const CbTile& tr = p.tiles[u.tile_lo + t];
        for (uint32_t c = 0; c < 16; ++c) {
          int64_t col = -1;
          if (p.aggregated) {
            const int64_t k = (int64_t)tr.xbase + c;
            if (k < p.cols_offset[tr.brow + 1]) col = p.restore_cols[k];
          } else {
            const int64_t k = (int64_t)tr.xbase + c;
            if (k < A.n) col = k;
          }
          g[16 * t + c] = (int32_t)col;
        }
      }
      if (!(p.lane_units[i].flags & CB_LUNIT_PLAINX)) compact_gather_list(p.lane_units[i], g);
      p.lane_units[i].flags |= span_max > CB_SCAN_SPAN ? CB_LUNIT_SCAN : 0;
    }
  });
  if (!moved.empty())
    for (uint32_t& sl : p.value_slot) sl = moved[sl];
  return CBSPMV_OK;
}

// Step 4a of the analysis: units of work over the tiles of p (p.tiles in block-row order,
// tile_off: nbr + 1 tile offsets of the block rows). Fills p.units (matrix order),
// p.split_rows, p.n_split_rows, p.n_split_wide and p.n_slots.
void cut_units(Plan& p, const std::vector<int64_t>& tile_off, const cbspmv_opts_t& opts, int n_workers) {
  const int64_t nbr = p.nbr;
  // Record layout: every unit must fit one warp's shared-memory
  // buffer (stream bytes, tiles, multiply-adds incl. Dense zero fill). Lane-stream layout:
  // the values stream through registers, so only the x slots (tiles) and rows bound a
  // unit, and its work is its stored entries.
  const bool lanes = p.lanes;
  const uint32_t BMAX = lanes ? UINT32_MAX : CB_B_MAX_FOR(p.vsize);   // stream bytes per unit
  // Lane-stream default: CB_LANE_WORK_DEFAULT entries per unit, smaller when that would
  // leave CTAs without a unit (a small matrix is then spread over all SMs), but never below
  // 256 entries or below the largest block row (so no block row is cut into more parts)
  uint32_t lane_default = CB_LANE_WORK_DEFAULT;
  if (lanes && opts.unit_work <= 0 && n_workers > 0 && p.nnz / CB_LANE_WORK_DEFAULT < n_workers) {
    int64_t wmax = 0;   // entries of the largest block row
    for (int64_t b = 0; b < nbr; ++b) {
      int64_t w = 0;
      for (int64_t t = tile_off[b]; t < tile_off[b + 1]; ++t) w += p.tiles[t].nnz;
      wmax = std::max(wmax, w);
    }
    lane_default = (uint32_t)std::min<int64_t>(CB_LANE_WORK_DEFAULT,
                                               std::max<int64_t>({int64_t{256}, wmax, p.nnz / n_workers}));
  }
  const uint32_t U = lanes ? (opts.unit_work > 0 ? std::min<uint32_t>((uint32_t)opts.unit_work, CB_LANE_WORK_MAX)
                                                 : lane_default)
                           : (opts.unit_work > 0 ? std::min<uint32_t>((uint32_t)opts.unit_work, CB_UNIT_WORK_MAX)
                                                 : CB_UNIT_WORK_DEFAULT);
  const int64_t TMAX = lanes ? CB_LANE_T_MAX : CB_T_MAX;
  const uint32_t NBRMAX = lanes ? CB_LANE_NBR_MAX : CB_NBR_MAX;
  auto tile_work = [&](int64_t t) -> uint32_t {
    return (!lanes && p.tiles[t].fmt == CB_FMT_DENSE) ? 256u : p.tiles[t].nnz;
  };
  auto tile_bytes = [&](int64_t t) -> uint32_t {
    return lanes ? 0u : record_bytes(p.tiles[t].fmt, p.tiles[t].nnz, p.vsize);
  };
  auto finish_unit = [&](CbUnit& u) {
    if (p.aggregated && u.ntiles > 0) {
      uint32_t first = p.tiles[u.tile_lo].xbase;
      uint32_t last = p.tiles[u.tile_lo + u.ntiles - 1].xbase + 16;
      u.rc_lo = first & ~3u;
      u.rc_n = (last - u.rc_lo + 3u) & ~3u;
    } else {
      u.rc_lo = 0;
      u.rc_n = 0;
    }
    if (u.ntiles > 0) u.byte_lo16 = p.tiles[u.tile_lo].vp16;
    p.units.push_back(u);
  };
  CbUnit open{};
  bool have_open = false;
  int32_t split_id = 0;
  uint32_t slot = 0;
  for (int64_t b = 0; b < nbr; ++b) {
    int64_t t0 = tile_off[b], t1 = tile_off[b + 1];
    uint64_t W = 0, B = 0;
    for (int64_t t = t0; t < t1; ++t) { W += tile_work(t); B += tile_bytes(t); }
    int64_t T = t1 - t0;
    bool big = W > U || B > BMAX || T > TMAX;
    if (!big) {
      if (have_open && open.work + W <= U && open.nbytes + B <= BMAX &&
          open.ntiles + T <= TMAX && open.nbr < NBRMAX) {
        open.ntiles = (uint16_t)(open.ntiles + T);
        open.nbr = (uint16_t)(open.nbr + 1);
        open.nbytes += (uint32_t)B;
        open.work += (uint32_t)W;
        if (open.ntiles == T) open.tile_lo = (uint32_t)t0;
        continue;
      }
      if (have_open) finish_unit(open);
      open = CbUnit{};
      open.tile_lo = (uint32_t)t0;
      open.ntiles = (uint16_t)T;
      open.nbr = 1;
      open.brow_lo = (uint32_t)b;
      open.nbytes = (uint32_t)B;
      open.work = (uint32_t)W;
      open.split = -1;
      open.nparts = 1;
      have_open = true;
      continue;
    }
    if (have_open) { finish_unit(open); have_open = false; }
    // cut the block row into parts of about equal work within the unit limits
    uint64_t nparts_est = std::max<uint64_t>({(W + U - 1) / U, (B + BMAX - 1) / BMAX,
                                              (uint64_t)((T + TMAX - 1) / TMAX), 2});
    uint64_t target = (W + nparts_est - 1) / nparts_est;
    size_t first_unit = p.units.size();
    CbUnit u{};
    u.tile_lo = (uint32_t)t0; u.nbr = 1; u.brow_lo = (uint32_t)b; u.split = split_id;
    for (int64_t t = t0; t < t1; ++t) {
      uint32_t wt = tile_work(t), bt = tile_bytes(t);
      if (u.ntiles > 0 && (u.work + wt > U || u.nbytes + bt > BMAX || u.ntiles + 1 > TMAX ||
                           u.work >= target)) {
        finish_unit(u);
        CbUnit v{};
        v.tile_lo = (uint32_t)t; v.nbr = 1; v.brow_lo = (uint32_t)b; v.split = split_id;
        u = v;
      }
      u.ntiles++;
      u.work += wt;
      u.nbytes += bt;
    }
    finish_unit(u);
    uint16_t np = (uint16_t)(p.units.size() - first_unit);
    CbSplitRow sr{};
    sr.slot0 = slot;
    sr.brow = (uint32_t)b;
    sr.nparts = np;
    sr.rows = (uint16_t)std::min<int64_t>(CB_BLK, p.m - b * CB_BLK);
    p.split_rows.push_back(sr);
    for (size_t i = first_unit; i < p.units.size(); ++i) {
      p.units[i].part = (uint16_t)(i - first_unit);
      p.units[i].nparts = np;
      p.units[i].slot = slot++;
    }
    ++split_id;
  }
  if (have_open) finish_unit(open);
  p.n_split_rows = split_id;
  // split rows with many parts last (they are added by a wider combine)
  std::stable_partition(p.split_rows.begin(), p.split_rows.end(),
                        [](const CbSplitRow& r) { return r.nparts <= CB_COMBINE_WIDE_PARTS; });
  p.n_split_wide = 0;
  for (const CbSplitRow& r : p.split_rows) p.n_split_wide += r.nparts > CB_COMBINE_WIDE_PARTS;
  p.n_slots = (int)slot;
}

// Every unit must fit the run kernel's buffers (the shared-memory stage of the record
// kernel, the step and row limits of the lane kernel).
cbspmv_status_t check_units(const Plan& p, std::string* msg) {
  const bool lanes = p.lanes;
  const uint32_t BMAX = lanes ? UINT32_MAX : CB_B_MAX_FOR(p.vsize);
  for (const CbUnit& u : p.units) {
    const bool bad = lanes ? (u.ntiles > CB_LANE_T_MAX || (u.work + 31) / 32 > 0xffffu ||
                              u.nbr > CB_LANE_NBR_MAX || u.nbr == 0)
                           : (u.nbytes > BMAX || u.ntiles > CB_T_MAX || u.rc_n > CB_RC_MAX ||
                              u.sched_bytes > CB_SCHED_MAX ||
                              u.blob_bytes > 16u * CB_T_MAX + 4u * CB_RC_MAX + CB_SCHED_MAX ||
                              u.nbr > CB_NBR_MAX || u.nbr == 0);
    if (bad) {
      *msg = "internal error: a unit exceeds the run kernel buffer limits";
      return CBSPMV_ERR_INVALID;
    }
  }
  return CBSPMV_OK;
}

// Step 4b: load balance of the units over the persistent thread blocks (Sec. 3.4):
// longest-processing-time order, min-heap of (load, worker id). Reorders p.units into
// worker order and fills p.worker_units, p.worker_off and *load_out (cost per worker).
void balance_units(Plan& p, const cbspmv_opts_t& opts, int n_workers, std::vector<double>* load_out) {
  const bool lanes = p.lanes;
  const int64_t nu = (int64_t)p.units.size();
  p.n_workers = n_workers;
  std::vector<double> cost(nu);
  for (int64_t i = 0; i < nu; ++i) {
    const CbUnit& u = p.units[i];
    // lane-stream units: the FP64 FMA slots of the walk (32 per step) plus the gather
    cost[i] = lanes ? 32.0 * ((u.work + 31) / 32) + 16.0 * u.ntiles + 2.0 * CB_BLK * u.nbr + 64.0
                    : (double)u.work + 8.0 * u.ntiles + 2.0 * CB_BLK * u.nbr + 64.0;
  }
  std::vector<std::vector<uint32_t>> lists(n_workers);
  std::vector<double>& load = *load_out;
  load.assign(n_workers, 0.0);
  if (opts.load_balance) {
    std::vector<uint32_t> order(nu);
    for (int64_t i = 0; i < nu; ++i) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
    typedef std::pair<double, int> Item;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    for (int w = 0; w < n_workers; ++w) pq.push(Item(0.0, w));
    for (uint32_t u : order) {
      Item top = pq.top();
      pq.pop();
      lists[top.second].push_back(u);
      top.first += cost[u];
      load[top.second] = top.first;
      pq.push(top);
    }
    for (auto& l : lists) std::sort(l.begin(), l.end());   // matrix order inside a worker
  } else {
    for (int64_t i = 0; i < nu; ++i) {
      lists[i % n_workers].push_back((uint32_t)i);
      load[i % n_workers] += cost[i];
    }
  }
  // store the units in worker order: each CTA's units are one contiguous range
  p.worker_off.assign(n_workers + 1, 0);
  p.worker_units.reserve(nu);
  for (int w = 0; w < n_workers; ++w) {
    p.worker_off[w + 1] = p.worker_off[w] + (uint32_t)lists[w].size();
    p.worker_units.insert(p.worker_units.end(), lists[w].begin(), lists[w].end());
  }
  {
    std::vector<CbUnit> ordered(nu);
    static_assert(sizeof(CbUnit) == 64, "unit descriptor is 64 bytes");
    for (int64_t i = 0; i < nu; ++i) ordered[i] = p.units[p.worker_units[i]];
    p.units.swap(ordered);
  }
}

// Statistics of a finished plan (analysis time excepted): plain_tiles and frac are the
// plain 16x16 tile count and super-sparse share of step 2, load the cost per worker.
void fill_stats(Plan& p, int64_t plain_tiles, double frac, const std::vector<double>& load) {
  const bool lanes = p.lanes;
  const int64_t nbr = p.nbr;
  const int64_t ntiles = (int64_t)p.tiles.size();
  const int n_workers = p.n_workers;
  const int64_t nu = (int64_t)p.units.size();
  cbspmv_stats_t& s = p.stats;
  s = cbspmv_stats_t{};
  s.m = p.m; s.n = p.n; s.nnz = p.nnz;
  s.n_block_rows = nbr;
  s.n_tiles = ntiles;
  s.n_tiles_plain = plain_tiles;
  s.super_sparse_fraction = frac;
  s.aggregated = p.aggregated ? 1 : 0;
  s.value_dtype = p.value_dtype;
  int64_t mults = 0;
  for (int64_t t = 0; t < ntiles; ++t) {
    const CbTile& x = p.tiles[t];
    s.n_fmt[x.fmt]++;
    s.nnz_fmt[x.fmt] += x.nnz;
    s.hist_coarse[std::min(7, (x.nnz - 1) / 32)]++;
    if (x.nnz <= 32) s.hist_fine[(x.nnz - 1) / 8]++;
    mults += x.fmt == CB_FMT_DENSE ? 256 : x.nnz;
  }
  s.restore_cols_len = p.restore_cols_len;
  if (lanes) {
    s.stream_bytes = (int64_t)p.n_lane_vals * p.vsize + (int64_t)p.n_lane_words * 8;
    s.metadata_bytes = ntiles * (int64_t)sizeof(CbTile) + (int64_t)p.n_lane_gcols * 4 +
                       (int64_t)p.lane_units.size() * (int64_t)sizeof(CbLaneUnit);
  } else {
    s.stream_bytes = (int64_t)p.stream.size();
    s.metadata_bytes = ntiles * (int64_t)sizeof(CbTile) + (int64_t)p.sched.size() * 4 +
                       (int64_t)p.units.size() * (int64_t)sizeof(CbUnit);
  }
  s.lane_layout = lanes ? 1 : 0;
  s.model_bytes_cb = ntiles * 21 + p.nnz * 9;
  s.model_bytes_csr = (p.m + 1) * 4 + p.nnz * 12;
  s.model_bytes_bsr16 = 2048 * ntiles + (nbr + 1) * 4 + 4 * ntiles;
  const int64_t es = p.value_dtype == CBSPMV_F64 ? 8 : 4;   // x, y element size
  s.algo_bytes_per_run = p.nnz * (int64_t)(p.vsize + 1) + ntiles * 21 + p.n * es + p.m * es +
                         (p.aggregated ? 4 * p.restore_cols_len : 0);
  s.flops_per_run = 2 * p.nnz;
  s.mults_per_run = mults;
  s.n_units = nu;
  int64_t nsplit_units = 0;
  for (auto& u : p.units) nsplit_units += u.split >= 0;
  s.n_split_units = nsplit_units;
  for (auto& u : p.units) {
    s.n_entry_mode_units += (u.mode & CB_MODE_ENTRY) ? 1 : 0;
    s.n_xseq_units += (u.mode & CB_MODE_XSEQ) ? 1 : 0;
    s.n_direct_units += (u.mode & CB_MODE_DIRECT) ? 1 : 0;
  }
  s.fma_slots = p.fma_slots;
  for (const CbLaneUnit& L : p.lane_units) {
    const bool plainx = (L.flags & CB_LUNIT_PLAINX) != 0, g16 = (L.flags & CB_LUNIT_G16) != 0;
    s.n_g16_units += g16 ? 1 : 0;
    s.gather_list_bytes += plainx ? 4 * (int64_t)((L.nslots / 16 + 3) / 4 * 4) : (g16 ? 2 : 4) * (int64_t)L.nslots;
  }
  s.n_split_rows = p.n_split_rows;
  s.n_workers = n_workers;
  double lmax = 0, lsum = 0, lsq = 0;
  for (double l : load) { lmax = std::max(lmax, l); lsum += l; lsq += l * l; }
  s.worker_load_max = lmax;
  s.worker_load_mean = lsum / n_workers;
  s.worker_load_std = std::sqrt(std::max(0.0, lsq / n_workers - s.worker_load_mean * s.worker_load_mean));
  {
    int64_t ng = (ntiles + 7) / 8;
    double gs = 0, gq = 0;
    for (int64_t g = 0; g < ng; ++g) {
      double v = 0;
      for (int64_t t = 8 * g; t < std::min(ntiles, 8 * g + 8); ++t) v += p.tiles[t].nnz;
      gs += v; gq += v * v;
    }
    double mean = ng ? gs / ng : 0;
    s.tb8_load_std = ng ? std::sqrt(std::max(0.0, gq / ng - mean * mean)) : 0.0;
  }
}

// Options shared by the host and the device analysis.
cbspmv_status_t check_opts(const cbspmv_opts_t& opts, int n_workers, std::string* msg) {
  if (opts.th1 < 0 || opts.th2 < opts.th1 || opts.th2 > 256 || !(opts.th0 >= 0.0)) {
    *msg = "thresholds must satisfy th0 >= 0 and 0 <= th1 <= th2 <= 256";
    return CBSPMV_ERR_INVALID;
  }
  if (opts.value_dtype < CBSPMV_F64 || opts.value_dtype > CBSPMV_F16) {
    *msg = "unknown value_dtype";
    return CBSPMV_ERR_INVALID;
  }
  if (opts.col_agg < -1 || opts.col_agg > 1) { *msg = "col_agg must be -1, 0 or 1"; return CBSPMV_ERR_INVALID; }
  if (opts.keep_value_map != 0 && opts.keep_value_map != 1) { *msg = "keep_value_map must be 0 or 1"; return CBSPMV_ERR_INVALID; }
  if (opts.record_layout < 0 || opts.record_layout > 2) { *msg = "record_layout must be 0, 1 or 2"; return CBSPMV_ERR_INVALID; }
  if (opts.plain_records != 0 && opts.plain_records != 1) { *msg = "plain_records must be 0 or 1"; return CBSPMV_ERR_INVALID; }
  if (n_workers <= 0) { *msg = "no workers"; return CBSPMV_ERR_INVALID; }
  return CBSPMV_OK;
}

cbspmv_status_t analyze_host(const cbspmv_csr_t& A, const cbspmv_opts_t& opts, int n_workers,
                             Plan* P, std::string* msg) {
  auto t_start = std::chrono::steady_clock::now();
  cbspmv_status_t st = check_opts(opts, n_workers, msg);
  if (st != CBSPMV_OK) return st;
  st = validate(A, msg);
  if (st != CBSPMV_OK) return st;

  Plan& p = *P;
  p = Plan();
  p.m = A.m; p.n = A.n; p.nnz = A.nnz;
  p.nbr = (A.m + CB_BLK - 1) / CB_BLK;
  p.value_dtype = opts.value_dtype;
  p.vsize = value_size(opts.value_dtype);
  p.th0 = opts.th0; p.th1 = opts.th1; p.th2 = opts.th2;
  p.lanes = uses_lanes(opts);
  const int64_t nbr = p.nbr;

  // --- step 2: plain 16x16 tiles and the super-sparse share (Sec. 3.3.1)
  std::atomic<int64_t> plain_tiles(0), plain_sparse(0);
  parallel_for(nbr, 256, [&](int64_t lo, int64_t hi) {
    std::vector<uint32_t> bj, tmp;
    int64_t pt = 0, ps = 0;
    for (int64_t b = lo; b < hi; ++b) {
      bj.clear();
      int64_t r0 = b * CB_BLK, r1 = std::min<int64_t>(A.m, r0 + CB_BLK);
      size_t bounds[CB_BLK + 1];
      int nr = 0;
      bounds[0] = 0;
      for (int64_t r = r0; r < r1; ++r) {
        for (int64_t k = A.row_ptr[r]; k < A.row_ptr[r + 1]; ++k) bj.push_back((uint32_t)A.col_idx[k] >> 4);
        bounds[++nr] = bj.size();
      }
      merge_sorted_runs(bj, tmp, bounds, nr);   // each row's block columns ascend
      size_t i = 0;
      while (i < bj.size()) {
        size_t j = i;
        while (j < bj.size() && bj[j] == bj[i]) ++j;
        ++pt;
        if ((int64_t)(j - i) < opts.th1) ++ps;
        i = j;
      }
    }
    plain_tiles += pt;
    plain_sparse += ps;
  });
  double frac = plain_tiles.load() ? (double)plain_sparse.load() / (double)plain_tiles.load() : 0.0;
  p.aggregated = opts.col_agg < 0 ? (frac > opts.th0) : (opts.col_agg == 1);

  // --- step 3: per block row aggregation, tiling, format selection and packing
  std::vector<BlockRowOut> rows(nbr);
  parallel_for(nbr, 64, [&](int64_t lo, int64_t hi) {
    std::vector<std::pair<uint64_t, int64_t>> e, tmp;
    for (int64_t b = lo; b < hi; ++b)
      build_block_row(A, b, p.aggregated, opts.th1, opts.th2, p.value_dtype, opts.keep_value_map != 0, e, tmp,
                      rows[b]);
  });
  // prefix sums over block rows: tiles, stream bytes, distinct columns
  std::vector<int64_t> tile_off(nbr + 1, 0), byte_off(nbr + 1, 0);
  p.cols_offset.assign(p.aggregated ? nbr + 1 : 0, 0);
  for (int64_t b = 0; b < nbr; ++b) {
    tile_off[b + 1] = tile_off[b] + (int64_t)rows[b].off.size();
    byte_off[b + 1] = byte_off[b] + (int64_t)rows[b].bytes.size();
    if (p.aggregated) p.cols_offset[b + 1] = p.cols_offset[b] + (int64_t)rows[b].distinct.size();
  }
  const int64_t ntiles = tile_off[nbr];
  if (byte_off[nbr] / 16 >= (1LL << 32)) { *msg = "packed stream exceeds 64 GiB"; return CBSPMV_ERR_UNSUPPORTED; }
  if (opts.keep_value_map && byte_off[nbr] / p.vsize >= (1LL << 32)) {
    *msg = "packed stream too large for a value map";
    return CBSPMV_ERR_UNSUPPORTED;
  }
  if (opts.keep_value_map) {
    try {
      p.value_slot.assign((size_t)A.nnz, 0);
    } catch (...) {
      *msg = "host allocation failed";
      return CBSPMV_ERR_OOM;
    }
  }
  p.restore_cols_len = p.aggregated ? p.cols_offset[nbr] : 0;
  std::vector<uint8_t> rowcnt;
  try {
    rowcnt.resize((size_t)ntiles * 16);
    p.tiles.resize(ntiles);
    p.tile_bcol.resize(ntiles);
    p.stream.resize(byte_off[nbr]);
    p.restore_cols.assign(p.restore_cols_len + CB_RC_PAD, 0);
  } catch (...) {
    *msg = "host allocation failed";
    return CBSPMV_ERR_OOM;
  }
  parallel_for(nbr, 256, [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; ++b) {
      BlockRowOut& o = rows[b];
      if (!o.bytes.empty()) std::memcpy(p.stream.data() + byte_off[b], o.bytes.data(), o.bytes.size());
      for (size_t i = 0; i < o.off.size(); ++i) {
        CbTile t{};
        t.vp16 = (uint32_t)((byte_off[b] + o.off[i]) / 16);
        t.xbase = p.aggregated ? (uint32_t)(p.cols_offset[b] + 16 * (int64_t)o.bcol[i]) : (uint32_t)(16 * o.bcol[i]);
        t.brow = (uint32_t)b;
        t.nnz = o.nnz[i];
        t.fmt = o.fmt[i];
        p.tiles[tile_off[b] + i] = t;
        p.tile_bcol[tile_off[b] + i] = o.bcol[i];
      }
      if (p.aggregated && !o.distinct.empty())
        std::memcpy(p.restore_cols.data() + p.cols_offset[b], o.distinct.data(), o.distinct.size() * 4);
      if (!o.rowcnt.empty()) std::memcpy(rowcnt.data() + (size_t)tile_off[b] * 16, o.rowcnt.data(), o.rowcnt.size());
      for (const auto& vs : o.vslot) p.value_slot[vs.first] = (uint32_t)((byte_off[b] + vs.second) / p.vsize);
      std::vector<std::pair<int64_t, uint32_t>>().swap(o.vslot);
      BlockRowOut().bytes.swap(o.bytes);
      std::vector<uint8_t>().swap(o.rowcnt);
    }
  });

  cut_units(p, tile_off, opts, n_workers);
  const bool lanes = p.lanes;
  const uint32_t BMAX = lanes ? UINT32_MAX : CB_B_MAX_FOR(p.vsize);

  // --- step 4a': lane schedule of every unit (chunks of <= CB_CHUNK entries, see cb_layout.h)
  if (!lanes) {
    const size_t nun = p.units.size();
    // bytes of each unit's schedule: header + steps * 64
    std::vector<uint64_t> sbytes(nun), chunks_of(nun);
    parallel_for((int64_t)nun, 256, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        const CbUnit& u = p.units[i];
        const int64_t R = std::min<int64_t>((int64_t)CB_BLK * u.nbr, A.m - (int64_t)u.brow_lo * CB_BLK);
        uint64_t nch = 0, nent = 0, nchx = 0;
        for (uint32_t t = 0; t < u.ntiles; ++t) {
          const size_t tg = (size_t)(u.tile_lo + t);
          const int64_t brl = (int64_t)p.tiles[tg].brow - u.brow_lo;
          uint32_t s0 = 0;
          for (int rr = 0; rr < 16; ++rr) {
            const uint32_t c = rowcnt[tg * 16 + rr];
            if (brl * 16 + rr < R) {
              nch += (c + CB_CHUNK - 1) / CB_CHUNK;
              nent += c;
              nchx += xseq_chunks(p, tg, rr, s0, c);
            }
            s0 += c;
          }
        }
        // Schedule mode (see cb_layout.h): consecutive-column chunks when they fill their
        // FMA slots about as well as plain chunks; plain chunks; single entries for sparse
        // pieces (CB_ENTRY_MODE_FILL).
        const double fill3 = nch ? (double)nent / (CB_CHUNK * (double)nch) : 0.0;
        const double fillx = nchx ? (double)nent / (CB_CHUNK * (double)nchx) : 0.0;
        uint32_t mode = 0;
        if (nch > 0 && fillx >= CB_ENTRY_MODE_FILL && fillx >= 0.9 * fill3) {
          mode = CB_MODE_XSEQ;
          nch = nchx;
        } else if (nch > 0 && fill3 < CB_ENTRY_MODE_FILL) {
          mode = CB_MODE_ENTRY;
          nch = nent;
        }
        // Direct descriptors where the chunks' columns are known per chunk: two fewer
        // dependent shared-memory loads per chunk for twice the descriptor bytes, and the
        // unit's values re-laid in load order (below).
        if ((mode & (CB_MODE_ENTRY | CB_MODE_XSEQ)) && nch <= CB_DIRECT_MAX_CHUNKS && !opts.plain_records)
          mode |= CB_MODE_DIRECT;
        p.units[i].mode = mode;
        chunks_of[i] = nch;
        // descriptor rows: chunks of the longest run, rounded up to an even count because
        // the kernel reads the chunks of a run in pairs
        const uint64_t rows = ((nch + CB_VLANES - 1) / CB_VLANES + 1) & ~1ULL;
        sbytes[i] = CB_SCHED_HDR(R) + ((mode & CB_MODE_DIRECT) ? 4 : 2) * CB_VLANES * rows;
      }
    });
    std::vector<uint64_t> off(nun + 1, 0);
    for (size_t i = 0; i < nun; ++i) off[i + 1] = off[i] + sbytes[i];
    // every lane of a unit's warp runs (descriptor rows) chunk steps of (chunk size) slots
    p.fma_slots = 0;
    for (size_t i = 0; i < nun; ++i) {
      const uint64_t rows = ((chunks_of[i] + CB_VLANES - 1) / CB_VLANES + 1) & ~1ULL;
      const uint64_t cap = (p.units[i].mode & CB_MODE_ENTRY) ? 1u : (uint64_t)CB_CHUNK;
      p.fma_slots += (int64_t)(CB_VLANES * rows * cap);
    }
    if (off[nun] / 16 >= (1ULL << 32)) { *msg = "schedule array too large"; return CBSPMV_ERR_UNSUPPORTED; }
    p.sched.resize(off[nun] / 4);   // zeroed unit by unit below (descriptors past a run's end are 0)
    // new value slot of every value slot a direct unit re-lays (only for the value map)
    std::vector<uint32_t> moved(p.value_slot.empty() ? 0 : p.stream.size() / p.vsize, UINT32_MAX);
    parallel_for((int64_t)nun, 128, [&](int64_t lo, int64_t hi) {
      std::vector<uint16_t> chunk;      // descriptors in row-major order
      std::vector<uint32_t> chunk32;    // direct descriptors (CB_MODE_DIRECT units)
      std::vector<uint8_t> old;         // a direct unit's stream bytes before re-laying
      std::vector<uint8_t> chunk_row;   // row of each chunk
      std::vector<uint8_t> chunk_first; // chunk starts its row
      for (int64_t i = lo; i < hi; ++i) {
        CbUnit& u = p.units[i];
        const int64_t R = std::min<int64_t>((int64_t)CB_BLK * u.nbr, A.m - (int64_t)u.brow_lo * CB_BLK);
        uint8_t* base = reinterpret_cast<uint8_t*>(p.sched.data()) + off[i];
        std::memset(base, 0, sbytes[i]);
        uint16_t* hdr = reinterpret_cast<uint16_t*>(base);
        uint8_t* nxt = base + 2 * CB_VLANES;
        uint16_t* desc = reinterpret_cast<uint16_t*>(base + CB_SCHED_HDR(R));
        chunk.clear(); chunk32.clear(); chunk_row.clear(); chunk_first.clear();
        const bool direct = (u.mode & CB_MODE_DIRECT) != 0;
        // tiles of each block row of the unit are consecutive; walk rows in order
        uint32_t t_begin = 0;
        for (int64_t brl = 0; brl < u.nbr; ++brl) {
          uint32_t t_end = t_begin;
          while (t_end < u.ntiles && (int64_t)p.tiles[u.tile_lo + t_end].brow - u.brow_lo == brl) ++t_end;
          for (int rr = 0; rr < 16; ++rr) {
            const int64_t row = brl * 16 + rr;
            if (row >= R) break;
            bool first = true;
            for (uint32_t t = t_begin; t < t_end; ++t) {
              const size_t tg = (size_t)(u.tile_lo + t);
              const uint32_t c = rowcnt[tg * 16 + rr];
              if (!c) continue;
              uint32_t s0;
              if (p.tiles[tg].fmt == CB_FMT_DENSE) {
                s0 = 16u * rr;
              } else {
                s0 = 0;
                for (int q = 0; q < rr; ++q) s0 += rowcnt[tg * 16 + q];
              }
              const uint32_t cap = (u.mode & CB_MODE_ENTRY) ? 1u : (uint32_t)CB_CHUNK;
              const bool xseq = (u.mode & CB_MODE_XSEQ) != 0;
              for (uint32_t o = 0; o < c;) {
                uint32_t len = std::min<uint32_t>(cap, c - o);
                if (xseq) len = xseq_run(p, tg, s0 + o, len);   // stop at a column gap
                chunk.push_back((uint16_t)(t | ((s0 + o) << 5) | (len << 13)));
                if (direct) {
                  const CbTile& tr = p.tiles[tg];
                  const uint32_t area = tr.fmt == CB_FMT_COO   ? align16(tr.nnz)
                                        : tr.fmt == CB_FMT_CSR ? align16(17u + tr.nnz)
                                                               : 32u;
                  const uint32_t voff = (tr.vp16 - u.byte_lo16) * 16u + area + (s0 + o) * (uint32_t)p.vsize;
                  chunk32.push_back((voff >> 1) | (t << 12) | (entry_col(p, tg, s0 + o) << 17) | (len << 21) |
                                    ((s0 + o) << 24));
                }
                chunk_row.push_back((uint8_t)row);
                chunk_first.push_back(first ? 1 : 0);
                first = false;
                o += len;
              }
            }
            if (!first) {                                      // last chunk of the row
              chunk.back() |= (uint16_t)0x8000u;
              if (direct) chunk32.back() |= 1u << 23;
            }
          }
          t_begin = t_end;
        }
        // next row holding entries, for every row
        {
          std::vector<uint8_t> has(R, 0);
          for (uint8_t r : chunk_row) has[r] = 1;
          int next = 0xff;
          for (int64_t r = R - 1; r >= 0; --r) {
            nxt[r] = (uint8_t)next;
            if (has[r]) next = (int)r;
          }
        }
        const uint64_t nch = chunk.size();
        if (direct) {
          // Re-lay the unit's stream bytes: the tiles' coordinate parts first (compacted,
          // 16-byte aligned), then the values in load order -- chunk index within a run,
          // then lane -- so that the lanes of one load instruction read consecutive bytes
          // instead of addresses one run length apart (which fall on few shared-memory
          // banks). The direct descriptors are retargeted; the coordinate parts keep the
          // record layout for export.
          const size_t ub = (size_t)u.byte_lo16 * 16;
          old.assign(p.stream.begin() + ub, p.stream.begin() + ub + u.nbytes);
          uint8_t* neu = p.stream.data() + ub;   // re-laid in place from the copy
          uint32_t w = 0;
          for (uint32_t t = 0; t < u.ntiles; ++t) {
            CbTile& tr = p.tiles[u.tile_lo + t];
            const uint32_t cpart = tr.fmt == CB_FMT_COO   ? align16(tr.nnz)
                                   : tr.fmt == CB_FMT_CSR ? align16(17u + tr.nnz)
                                                          : 32u;
            std::memcpy(neu + w, old.data() + ((size_t)tr.vp16 * 16 - ub), cpart);
            tr.vp16 = (uint32_t)((ub + w) / 16);
            w += cpart;
          }
          const uint32_t vs = (uint32_t)p.vsize;
          const uint64_t run_max = (nch + CB_VLANES - 1) / CB_VLANES;
          for (uint64_t j = 0; j < run_max; ++j)
            for (uint32_t l = 0; l < CB_VLANES; ++l) {
              const uint64_t c0 = (l * nch) / CB_VLANES, c1 = ((l + 1) * nch) / CB_VLANES;
              if (c0 + j >= c1) continue;
              uint32_t& d = chunk32[c0 + j];
              const uint32_t len = (d >> 21) & 3u, vo = (d & 0xfffu) << 1;
              std::memcpy(neu + w, old.data() + vo, (size_t)len * vs);
              if (!moved.empty())
                for (uint32_t q = 0; q < len; ++q) moved[(ub + vo) / vs + q] = (uint32_t)((ub + w) / vs + q);
              d = (d & ~0xfffu) | (w >> 1);
              w += len * vs;
            }
          std::memset(neu + w, 0, u.nbytes - w);   // the record padding the re-layout freed
        }
        int first_lane[CB_R_MAX], last_lane[CB_R_MAX];   // lanes holding chunks of each row
        for (int r = 0; r < CB_R_MAX; ++r) first_lane[r] = last_lane[r] = -1;
        for (uint32_t l = 0; l < CB_VLANES; ++l) {
          const uint64_t c0 = (l * nch) / CB_VLANES, c1 = ((l + 1) * nch) / CB_VLANES;
          if (c1 == c0) { hdr[l] = 0; continue; }
          const uint32_t hs = chunk_first[c0] ? 0u : 1u;
          hdr[l] = (uint16_t)(chunk_row[c0] | (hs << 8) | ((uint32_t)(c1 - c0) << 9));
          for (uint64_t k = c0; k < c1; ++k) {
            const uint64_t j = k - c0;      // pairs of chunks (2i, 2i + 1) side by side
            if (direct)
              reinterpret_cast<uint32_t*>(desc)[((j >> 1) * CB_VLANES + l) * 2 + (j & 1)] = chunk32[k];
            else
              desc[((j >> 1) * CB_VLANES + l) * 2 + (j & 1)] = chunk[k];
            const int r = chunk_row[k];
            if (first_lane[r] < 0) first_lane[r] = (int)l;
            last_lane[r] = (int)l;
          }
        }
        int span_max = 0;
        for (int r = 0; r < CB_R_MAX; ++r)
          if (first_lane[r] >= 0) span_max = std::max(span_max, last_lane[r] - first_lane[r] + 1);
        if (span_max > CB_SCAN_SPAN) u.mode |= CB_MODE_SCAN;
        u.sched16 = (uint32_t)(off[i] / 16);
        u.sched_bytes = (uint32_t)sbytes[i];
      }
    });
    if (!moved.empty())
      for (uint32_t& s : p.value_slot)
        if (moved[s] != UINT32_MAX) s = moved[s];
  }

  // --- unit blobs: tile records, restore_cols slice and schedule of each unit, back to back
  if (!lanes) {
    const size_t nun = p.units.size();
    std::vector<uint64_t> boff(nun + 1, 0);
    for (size_t i = 0; i < nun; ++i) {
      CbUnit& u = p.units[i];
      u.blob_bytes = 16u * u.ntiles + 4u * u.rc_n + u.sched_bytes;
      boff[i + 1] = boff[i] + u.blob_bytes;
    }
    if (boff[nun] / 16 >= (1ULL << 32)) { *msg = "unit blob array too large"; return CBSPMV_ERR_UNSUPPORTED; }
    p.blob.resize(boff[nun]);       // tile records + restore_cols slice + schedule fill each blob
    parallel_for((int64_t)nun, 256, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        CbUnit& u = p.units[i];
        uint8_t* d = p.blob.data() + boff[i];
        if (u.ntiles) std::memcpy(d, p.tiles.data() + u.tile_lo, 16u * u.ntiles);
        if (u.rc_n) std::memcpy(d + 16u * u.ntiles, p.restore_cols.data() + u.rc_lo, 4u * u.rc_n);
        if (u.sched_bytes)
          std::memcpy(d + 16u * u.ntiles + 4u * u.rc_n, reinterpret_cast<const uint8_t*>(p.sched.data()) + (size_t)u.sched16 * 16,
                      u.sched_bytes);
        u.blob16 = (uint32_t)(boff[i] / 16);
      }
    });
  }

  st = check_units(p, msg);
  if (st != CBSPMV_OK) return st;

  std::vector<double> load;
  balance_units(p, opts, n_workers, &load);
  if (lanes) {
    st = build_lane_programs(A, p, rowcnt, msg);
    if (st != CBSPMV_OK) return st;
    cb::ByteBuf().swap(p.stream);   // the record stream is not part of the lane-stream layout
  }

  fill_stats(p, plain_tiles.load(), frac, load);
  p.stats.analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return CBSPMV_OK;
}

cbspmv_status_t decode_to_csr(int64_t m, int64_t n, int dtype, bool aggregated,
                              const std::vector<CbTile>& tiles, const std::vector<CbUnit>& units,
                              const uint8_t* blob, size_t blob_size, const uint8_t* stream,
                              size_t stream_size, const int32_t* restore_cols, size_t restore_len,
                              int64_t* row_ptr, int32_t* col, double* val, int64_t nnz_expected,
                              std::string* msg) {
  if (dtype < CBSPMV_F64 || dtype > CBSPMV_F16) { *msg = "unknown value type"; return CBSPMV_ERR_INVALID; }
  const int vsize = value_size(dtype);
  std::vector<int64_t> cnt(m + 1, 0);
  // Direct units keep their values in load order after the coordinate parts: the stream
  // offset of every value of their tiles, from the direct descriptors (first entry, length,
  // value offset) of the unit's lane schedule.
  std::vector<int64_t> vfirst(tiles.size(), -1);   // tile -> first slot in vpos
  std::vector<uint64_t> vunit(tiles.size(), 0);    // tile -> stream offset of its unit
  std::vector<uint16_t> vpos;                      // value offset inside the unit (< CB_B_MAX)
  for (const CbUnit& u : units) {
    if (!(u.mode & CB_MODE_DIRECT)) continue;
    const int64_t R = std::min<int64_t>((int64_t)CB_BLK * u.nbr, m - (int64_t)u.brow_lo * CB_BLK);
    const size_t so = (size_t)u.blob16 * 16 + 16u * u.ntiles + 4u * u.rc_n;
    if (R <= 0 || so + u.sched_bytes > blob_size || u.sched_bytes < CB_SCHED_HDR(R)) {
      *msg = "corrupt unit schedule";
      return CBSPMV_ERR_INVALID;
    }
    for (uint32_t t = 0; t < u.ntiles; ++t) {
      const CbTile& tr = tiles[u.tile_lo + t];
      vfirst[u.tile_lo + t] = (int64_t)vpos.size();
      vunit[u.tile_lo + t] = (uint64_t)u.byte_lo16 * 16;
      vpos.resize(vpos.size() + (tr.fmt == CB_FMT_DENSE ? 256u : tr.nnz), UINT16_MAX);
    }
    const uint32_t* d = reinterpret_cast<const uint32_t*>(blob + so + CB_SCHED_HDR(R));
    const size_t nd = (u.sched_bytes - CB_SCHED_HDR(R)) / 4;
    for (size_t k = 0; k < nd; ++k) {
      const uint32_t len = (d[k] >> 21) & 3u, t = (d[k] >> 12) & 31u, e = d[k] >> 24;
      if (!len) continue;
      const uint32_t vo_rel = (d[k] & 0xfffu) << 1;
      const uint64_t vo = (uint64_t)u.byte_lo16 * 16 + vo_rel;
      if (t >= u.ntiles) {
        *msg = "corrupt direct descriptor";
        return CBSPMV_ERR_INVALID;
      }
      const CbTile& tr = tiles[u.tile_lo + t];
      const uint32_t cap = tr.fmt == CB_FMT_DENSE ? 256u : tr.nnz;
      if (e + len > cap || vo + (uint64_t)len * vsize > stream_size) {
        *msg = "corrupt direct descriptor";
        return CBSPMV_ERR_INVALID;
      }
      for (uint32_t q = 0; q < len; ++q) vpos[vfirst[u.tile_lo + t] + e + q] = (uint16_t)(vo_rel + q * vsize);
    }
  }
  auto value_at = [&](size_t ti, uint32_t e, const uint8_t* plain) -> const uint8_t* {
    if (vfirst[ti] < 0) return plain;
    const uint16_t p = vpos[vfirst[ti] + e];
    return p == UINT16_MAX ? nullptr : stream + vunit[ti] + p;
  };
  auto for_entries = [&](size_t ti, const std::function<void(int64_t, int64_t, const uint8_t*)>& f) -> bool {
    const CbTile& t = tiles[ti];
    size_t off = (size_t)t.vp16 * 16;
    uint32_t rb = record_bytes(t.fmt, t.nnz, vsize);
    if (off + rb > stream_size) return false;
    const uint8_t* rec = stream + off;
    auto colof = [&](uint32_t lc, int64_t* c) -> bool {
      if (aggregated) {
        size_t i = (size_t)t.xbase + lc;
        if (i >= restore_len) return false;
        *c = restore_cols[i];
      } else {
        *c = (int64_t)t.xbase + lc;
      }
      return *c >= 0 && *c < n;
    };
    if (t.fmt == CB_FMT_DENSE) {
      for (uint32_t pos = 0; pos < 256; ++pos) {
        if (!(rec[pos >> 3] & (1u << (pos & 7)))) continue;
        int64_t r = (int64_t)t.brow * 16 + (pos >> 4), c;
        const uint8_t* v = value_at(ti, pos, rec + 32 + pos * vsize);
        if (r >= m || !colof(pos & 15u, &c) || !v) return false;
        f(r, c, v);
      }
    } else {
      const uint8_t* idx = rec + (t.fmt == CB_FMT_CSR ? 17 : 0);
      uint32_t voff = align16((uint32_t)(idx - rec) + t.nnz);
      for (uint32_t i = 0; i < t.nnz; ++i) {
        int64_t r = (int64_t)t.brow * 16 + (idx[i] & 15u), c;
        const uint8_t* v = value_at(ti, i, rec + voff + i * vsize);
        if (r >= m || !colof(idx[i] >> 4, &c) || !v) return false;
        f(r, c, v);
      }
    }
    return true;
  };
  for (size_t ti = 0; ti < tiles.size(); ++ti)
    if (!for_entries(ti, [&](int64_t r, int64_t, const uint8_t*) { cnt[r + 1]++; })) {
      *msg = "corrupt blocked layout";
      return CBSPMV_ERR_INVALID;
    }
  for (int64_t r = 0; r < m; ++r) cnt[r + 1] += cnt[r];
  if (cnt[m] != nnz_expected) { *msg = "entry count mismatch in blocked layout"; return CBSPMV_ERR_INVALID; }
  std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
  for (size_t ti = 0; ti < tiles.size(); ++ti)
    for_entries(ti, [&](int64_t r, int64_t c, const uint8_t* v) {
      int64_t k = cur[r]++;
      col[k] = (int32_t)c;
      val[k] = read_value(v, dtype);
    });
  std::memcpy(row_ptr, cnt.data(), (m + 1) * sizeof(int64_t));
  // tiles of a block row are in increasing column order, so rows come out sorted; check
  for (int64_t r = 0; r < m; ++r)
    for (int64_t k = row_ptr[r] + 1; k < row_ptr[r + 1]; ++k)
      if (col[k] <= col[k - 1]) { *msg = "blocked layout decodes to unsorted rows"; return CBSPMV_ERR_INVALID; }
  return CBSPMV_OK;
}

cbspmv_status_t decode_lanes_to_csr(int64_t m, int64_t n, int dtype, const std::vector<CbLaneUnit>& units,
                                    const uint8_t* vals, size_t nvals, const uint64_t* words, size_t nwords,
                                    const int32_t* gcols, size_t ngcols, int64_t* row_ptr, int32_t* col,
                                    double* val, int64_t nnz_expected, std::string* msg) {
  const int vs = value_size(dtype);
  const bool grouped = vs != 8;
  // every entry once: (global row, column, value), counted per row first
  std::vector<int64_t> cnt((size_t)m + 1, 0);
  auto for_each = [&](const std::function<bool(int64_t, int32_t, double)>& f) -> bool {
    for (const CbLaneUnit& u : units) {
      const size_t v0 = (size_t)u.vals * CB_VLANES, w0 = (size_t)u.words * CB_VLANES;
      const uint32_t S = u.steps;
      const bool plainx = (u.flags & CB_LUNIT_PLAINX) != 0, g16 = (u.flags & CB_LUNIT_G16) != 0;
      const uint32_t ng = plainx ? (u.nslots / 16 + 3) / 4 * 4 : u.nslots;
      if (v0 + (size_t)S * CB_VLANES > nvals || w0 + (size_t)((S + 3) / 4) * CB_VLANES > nwords ||
          (size_t)u.gcols + ng > ngcols)
        return false;
      const uint16_t* g16p = reinterpret_cast<const uint16_t*>(gcols + u.gcols);
      for (uint32_t s = 0; s < S; ++s)
        for (uint32_t l = 0; l < CB_VLANES; ++l) {
          const uint32_t w = (uint32_t)(words[w0 + cb_lane_word_index(grouped, s, l, S)] >> (16 * (s % 4))) & 0xffffu;
          if (w == CB_LANE_NONE) continue;
          const uint32_t slot = w & 511u, r = w >> 9;
          if (slot >= u.nslots || r >= u.nrows) return false;
          int64_t c;
          if (plainx) c = (int64_t)gcols[u.gcols + slot / 16] + slot % 16;
          else if (g16) c = g16p[slot] == 0xffffu ? -1 : (int64_t)u.gbase + g16p[slot];
          else c = (int64_t)gcols[u.gcols + slot];
          const int64_t row = (int64_t)u.brow_lo * CB_BLK + r;
          if (c < 0 || c >= n || row >= m) return false;
          if (!f(row, (int32_t)c, read_value(vals + (v0 + cb_lane_val_index(grouped, s, l, S)) * vs, dtype))) return false;
        }
    }
    return true;
  };
  int64_t total = 0;
  if (!for_each([&](int64_t r, int32_t, double) { cnt[(size_t)r + 1]++; ++total; return true; }) ||
      total != nnz_expected) {
    *msg = "lane stream is inconsistent with the matrix";
    return CBSPMV_ERR_INVALID;
  }
  for (int64_t r = 0; r < m; ++r) cnt[(size_t)r + 1] += cnt[(size_t)r];
  for (int64_t r = 0; r <= m; ++r) row_ptr[r] = cnt[(size_t)r];
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  std::vector<std::pair<int32_t, double>> tmp;
  for_each([&](int64_t r, int32_t c, double v) {
    const int64_t k = fill[(size_t)r]++;
    col[k] = c;
    val[k] = v;
    return true;
  });
  // entries of a row come from its units in worker order: sort each row by column
  for (int64_t r = 0; r < m; ++r) {
    const int64_t a = row_ptr[r], b = row_ptr[r + 1];
    tmp.resize((size_t)(b - a));
    for (int64_t k = a; k < b; ++k) tmp[(size_t)(k - a)] = {col[k], val[k]};
    std::sort(tmp.begin(), tmp.end(), [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
      return x.first < y.first;
    });
    for (int64_t k = a; k < b; ++k) {
      col[k] = tmp[(size_t)(k - a)].first;
      val[k] = tmp[(size_t)(k - a)].second;
      if (k > a && col[k] == col[k - 1]) {
        *msg = "lane stream holds an entry twice";
        return CBSPMV_ERR_INVALID;
      }
    }
  }
  return CBSPMV_OK;
}

}  // namespace cb
