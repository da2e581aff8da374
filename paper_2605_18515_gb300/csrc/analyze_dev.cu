// Device-side analysis of a CSR that already lives on the GPU (the preprocessing of Sec. 3.2
// to 3.4 whose cost Sec. 4.5 weighs against the products): the lane-stream layout of
// cb_layout.h is built from the device arrays without copying the matrix to the host.
//
// On the GPU:
//   1. the CSR checks (row_ptr non-decreasing; columns strictly increasing in [0, n)),
//   2. the sorted column multiset of every 16-row block row (the union of its 16 sorted
//      rows, duplicates kept): a warp merges a block row of at most kMergeCap entries in
//      shared memory (four levels of pairwise merges, every element placed by its rank in
//      the partner run); larger block rows are merged level by level in global memory, in
//      chunks of kBigChunk outputs per CTA located by merge-path co-ranks,
//   3. the plain 16x16 tile count and the super-sparse count of Sec. 3.3.1 (which decide
//      the column aggregation), then the tiles of every block row (plain block columns, or
//      groups of 16 distinct columns when aggregated) with their entry counts, and the
//      restore_cols array of the aggregated columns,
//   4. the lane programs of every unit (values, 16-bit entry words, gather lists and the
//      carry-scan flag), the same arrays the host analysis writes, and the value map.
// On the host, between them: the aggregation decision, the prefix sums over block rows,
// the units of work (Sec. 3.4's tile groups) and their load balance, from the tile entry
// counts only (cut_units / balance_units / lane_offsets, shared with the host analysis).
// The entries of a unit in lane order are its rows' CSR entries restricted to the unit's
// tiles, so the lane build reads the CSR directly and finds each entry's slot by binary
// search in the unit's gather list.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cbspmv.h"
#include "cb_analyze_dev.h"
#include "cb_layout.h"
#include "cb_plan.h"
#include "cb_round.h"

namespace cb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMergeWarps = 12;     // warps per CTA of the shared-memory merge
constexpr int kMergeCap = 2048;     // entries of a block row merged in shared memory
constexpr int kBigChunk = 2048;     // outputs per CTA of a global-memory merge level
constexpr int kBigThreads = 256;
constexpr int kLaneRows = CB_LANE_NBR_MAX * CB_BLK;   // rows of a lane-stream unit at most
constexpr int kBuildWarps = 8;

// error flags
constexpr uint32_t kErrRowPtr = 1u;
constexpr uint32_t kErrCols = 2u;
constexpr uint32_t kErrUnit = 4u;

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// first index i in [0, n) with a[i] >= x (n if none)
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// first index i in [0, n) with a[i] > x (n if none)
__device__ __forceinline__ int upper_bound_i32(const int32_t* a, int n, int32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// Number of A elements among the first d outputs of the stable merge of A and B (A first
// on ties): the merge-path co-rank.
__device__ __forceinline__ int corank(const int32_t* A, int la, const int32_t* B, int lb, int d) {
  int lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - mid - 1]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// (1a) row_ptr of every block row non-decreasing; block rows above kMergeCap entries are
// listed (in any order) for the global-memory merge.
__global__ void check_rows_kernel(const int64_t* __restrict__ rp, int64_t m, int64_t nbr, uint32_t* err,
                                  uint32_t* nbig, int32_t* big) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbr; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = b * CB_BLK, r1 = min(m, r0 + CB_BLK);
    int64_t prev = rp[r0];
    bool bad = false;
    for (int64_t r = r0 + 1; r <= r1; ++r) {
      const int64_t v = rp[r];
      bad |= v < prev;
      prev = v;
    }
    if (bad) atomicOr(err, kErrRowPtr);
    else if (prev - rp[r0] > kMergeCap) big[atomicAdd(nbig, 1u)] = (int32_t)b;
  }
}

// (1b) columns of every row strictly increasing and in [0, n); a warp per row. Runs only
// after row_ptr passed, so every read lies inside the column array.
__global__ void check_cols_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t m,
                                  int64_t n, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < m; r += nw) {
    const int64_t a = rp[r], z = rp[r + 1];
    int32_t carry = -1;
    bool bad = false;
    for (int64_t k0 = a; k0 < z; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t c = k < z ? col[k] : INT32_MAX;
      int32_t p = __shfl_up_sync(kFull, c, 1);
      if (lane == 0) p = carry;
      if (k < z) bad |= c <= p || (int64_t)c >= n;
      carry = __shfl_sync(kFull, c, 31);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, kErrCols);
  }
}

// (2a) sorted column multiset of every block row with at most kMergeCap entries, a warp
// per block row: the 16 sorted rows merge pairwise in four levels in shared memory; an
// element of the left run lands at its index plus the count of smaller elements of the
// right run, an element of the right run at its index plus the count of elements of the
// left run not above it.
__global__ void __launch_bounds__(32 * kMergeWarps) merge_small_kernel(const int64_t* __restrict__ rp,
                                                                      const int32_t* __restrict__ col, int64_t m,
                                                                      int64_t nbr, int32_t* __restrict__ merged) {
  extern __shared__ int32_t msm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* buf0 = msm + (size_t)warp * 2 * kMergeCap;
  int32_t* buf1 = buf0 + kMergeCap;
  const int64_t nw = (int64_t)gridDim.x * kMergeWarps;
  for (int64_t b = blockIdx.x * (int64_t)kMergeWarps + warp; b < nbr; b += nw) {
    const int64_t r0 = b * CB_BLK;
    const int nr = (int)imin64(CB_BLK, m - r0);
    const int64_t base = rp[r0];
    const int bnd = lane <= nr ? (int)(rp[r0 + lane] - base) : 0;   // run bounds, lane j: row j
    const int E = __shfl_sync(kFull, bnd, nr);
    if (E > kMergeCap) continue;   // merged in global memory
    for (int i = lane; i < E; i += 32) buf0[i] = col[base + i];
    __syncwarp();
    int32_t* src = buf0;
    int32_t* dst = buf1;
    for (int w = 1; w < CB_BLK; w *= 2) {
      for (int q = 0; q < CB_BLK; q += 2 * w) {
        const int a0 = __shfl_sync(kFull, bnd, min(q, nr));
        const int a1 = __shfl_sync(kFull, bnd, min(q + w, nr));
        const int b1 = __shfl_sync(kFull, bnd, min(q + 2 * w, nr));
        for (int i = a0 + lane; i < b1; i += 32) {
          const int32_t x = src[i];
          const int pos = i < a1 ? (i - a0) + lower_bound_i32(src + a1, b1 - a1, x)
                                 : (i - a1) + upper_bound_i32(src + a0, a1 - a0, x);
          dst[a0 + pos] = x;
        }
      }
      __syncwarp();
      int32_t* t = src;
      src = dst;
      dst = t;
    }
    for (int i = lane; i < E; i += 32) merged[base + i] = src[i];
    __syncwarp();
  }
}

// (2b) one level of the global-memory merge of the large block rows: every item merges
// kBigChunk outputs of one run pair (runs [a0, a0 + la) and [a0 + la, a0 + la + lb) of
// src into the same positions of dst).
__global__ void __launch_bounds__(kBigThreads) merge_big_kernel(const MergeItem* __restrict__ items, int nitems,
                                                               const int32_t* __restrict__ src,
                                                               int32_t* __restrict__ dst) {
  __shared__ int32_t sA[kBigChunk], sB[kBigChunk], sO[kBigChunk];
  __shared__ int s_i0, s_i1;
  constexpr int kPer = kBigChunk / kBigThreads;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const MergeItem w = items[it];
    const int32_t* A = src + w.a0;
    const int32_t* B = A + w.la;
    const int total = w.la + w.lb;
    const int d0 = w.d0, d1 = min(d0 + kBigChunk, total);
    if (threadIdx.x == 0) s_i0 = corank(A, w.la, B, w.lb, d0);
    if (threadIdx.x == 32) s_i1 = corank(A, w.la, B, w.lb, d1);
    __syncthreads();
    const int i0 = s_i0, i1 = s_i1;
    const int na = i1 - i0, nb = (d1 - i1) - (d0 - i0);
    for (int k = threadIdx.x; k < na; k += kBigThreads) sA[k] = A[i0 + k];
    for (int k = threadIdx.x; k < nb; k += kBigThreads) sB[k] = B[d0 - i0 + k];
    __syncthreads();
    const int dl = kPer * threadIdx.x;
    if (dl < na + nb) {
      int ia = corank(sA, na, sB, nb, dl), ib = dl - ia;
      for (int k = 0; k < kPer && dl + k < na + nb; ++k)
        sO[dl + k] = (ib >= nb || (ia < na && sA[ia] <= sB[ib])) ? sA[ia++] : sB[ib++];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < na + nb; k += kBigThreads) dst[w.a0 + d0 + k] = sO[k];
    __syncthreads();
  }
}

// Entries of the sorted block-row multiset stream through a warp 32 at a time. A "tile
// key" of an entry is its plain block column (col >> 4) or, when aggregated, its distinct
// column rank >> 4; a tile is a run of one key.
struct KeyScan {
  int64_t open_start = 0;   // entry index where the open tile starts
  int32_t prev_col = -1;    // last column of the previous chunk
  int32_t prev_key = -1;    // last key of the previous chunk
  int64_t ndist = 0;        // distinct columns so far
  int64_t ntiles = 0;       // tiles started so far
};

// (3a) plain tile count, super-sparse plain tiles (< th1 entries) and distinct columns of
// every block row (Sec. 3.3.1).
__global__ void tile_count_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ merged, int64_t m,
                                  int64_t nbr, int th1, int32_t* __restrict__ nplain, int32_t* __restrict__ ndist,
                                  unsigned long long* totals) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); b < nbr; b += nw) {
    const int64_t r0 = b * CB_BLK, r1 = min(m, r0 + CB_BLK);
    const int64_t base = rp[r0], E = rp[r1] - base;
    KeyScan s;
    int sparse = 0;
    for (int64_t c0 = 0; c0 < E; c0 += 32) {
      const int64_t i = c0 + lane;
      const bool valid = i < E;
      const int32_t x = valid ? merged[base + i] : INT32_MAX;
      int32_t xp = __shfl_up_sync(kFull, x, 1);
      if (lane == 0) xp = s.prev_col;
      const bool newd = valid && (i == 0 || x != xp);
      const bool newt = valid && (i == 0 || (x >> 4) != (xp >> 4));
      const unsigned md = __ballot_sync(kFull, newd), mt = __ballot_sync(kFull, newt);
      if (newt && i > 0) {   // the tile before this one closes at i
        const unsigned below = mt & lt;
        const int64_t start = below ? c0 + (31 - __clz(below)) : s.open_start;
        sparse += (i - start) < th1;
      }
      if (mt) s.open_start = c0 + (31 - __clz(mt));
      s.ndist += __popc(md);
      s.ntiles += __popc(mt);
      s.prev_col = __shfl_sync(kFull, x, 31);
    }
    if (lane == 0 && E > 0) sparse += (E - s.open_start) < th1;
    for (int o = 16; o; o >>= 1) sparse += __shfl_xor_sync(kFull, sparse, o);
    if (lane == 0) {
      nplain[b] = (int32_t)s.ntiles;
      ndist[b] = (int32_t)s.ndist;
      atomicAdd(totals + 0, (unsigned long long)s.ntiles);
      atomicAdd(totals + 1, (unsigned long long)sparse);
    }
  }
}

// (3b) tiles of every block row at tile_off[b]: entry count and block column (the key),
// and, when aggregated, the distinct columns at cols_off[b] (restore_cols).
__global__ void tile_write_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ merged, int64_t m,
                                  int64_t nbr, int agg, const int64_t* __restrict__ tile_off,
                                  const int64_t* __restrict__ cols_off, uint16_t* __restrict__ tnnz,
                                  int32_t* __restrict__ tkey, int32_t* __restrict__ rcols) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u, le = lt | (1u << lane);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); b < nbr; b += nw) {
    const int64_t r0 = b * CB_BLK, r1 = min(m, r0 + CB_BLK);
    const int64_t base = rp[r0], E = rp[r1] - base;
    const int64_t tb = tile_off[b], cb = agg ? cols_off[b] : 0;
    KeyScan s;
    for (int64_t c0 = 0; c0 < E; c0 += 32) {
      const int64_t i = c0 + lane;
      const bool valid = i < E;
      const int32_t x = valid ? merged[base + i] : INT32_MAX;
      int32_t xp = __shfl_up_sync(kFull, x, 1);
      if (lane == 0) xp = s.prev_col;
      const bool newd = valid && (i == 0 || x != xp);
      const unsigned md = __ballot_sync(kFull, newd);
      const int64_t rank = s.ndist + __popc(md & le) - 1;   // distinct rank of this column
      if (agg && newd) rcols[cb + rank] = x;
      const int32_t key = valid ? (agg ? (int32_t)(rank >> 4) : (x >> 4)) : INT32_MAX;
      int32_t kp = __shfl_up_sync(kFull, key, 1);
      if (lane == 0) kp = s.prev_key;
      const bool newt = valid && (i == 0 || key != kp);
      const unsigned mt = __ballot_sync(kFull, newt);
      if (newt && i > 0) {
        const unsigned below = mt & lt;
        const int64_t start = below ? c0 + (31 - __clz(below)) : s.open_start;
        const int64_t t = s.ntiles + __popc(mt & lt) - 1;   // index of the closing tile
        tnnz[tb + t] = (uint16_t)(i - start);
        tkey[tb + t] = kp;
      }
      if (mt) s.open_start = c0 + (31 - __clz(mt));
      s.ndist += __popc(md);
      s.ntiles += __popc(mt);
      s.prev_col = __shfl_sync(kFull, x, 31);
      const int last = (int)imin64(31, E - 1 - c0);
      s.prev_key = __shfl_sync(kFull, key, last);
    }
    if (lane == 0 && E > 0) {
      tnnz[tb + s.ntiles - 1] = (uint16_t)(E - s.open_start);
      tkey[tb + s.ntiles - 1] = s.prev_key;
    }
  }
}

// (4) lane programs of every unit, a warp per unit (layout in cb_layout.h). The gather list
// comes from the tiles' keys; each row's CSR entries, restricted to the unit's tiles (a
// split part of a block row holds a column range of it), are dealt to the 32 lanes in runs
// of floor(l W / 32), every entry's slot found by binary search in its block row's part of
// the gather list (ascending, with -1 padding only at the end of a block row's last tile).
struct LaneBuildArgs {
  const int64_t* rp;
  const int32_t* col;
  const double* val;
  int64_t m, n;
  int agg;
  const int64_t* tile_off;
  const int64_t* cols_off;
  const int32_t* tkey;
  const int32_t* rcols;
  CbLaneUnit* lunits;
  const uint32_t* utile;   // first tile of every unit
  uint32_t nunits;
  int dtype;               // storage type of the values
  uint8_t* lvals;
  uint64_t* lwords;
  int32_t* lgcols;
  uint32_t* vslot;         // value map (optional)
  uint32_t* err;
};

struct BuildSmem {
  int32_t g[CB_LANE_SLOTS];
  int32_t rlo[kLaneRows];
  int32_t e[kLaneRows + 1];
  int32_t tbl[CB_LANE_NBR_MAX], tbh[CB_LANE_NBR_MAX];
};

__global__ void __launch_bounds__(32 * kBuildWarps) lane_build_kernel(LaneBuildArgs a) {
  __shared__ BuildSmem sm_all[kBuildWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BuildSmem& w = sm_all[warp];
  const uint32_t nw = gridDim.x * kBuildWarps;
  for (uint32_t u = blockIdx.x * kBuildWarps + warp; u < a.nunits; u += nw) {
    const CbLaneUnit L = a.lunits[u];
    const uint32_t tlo = a.utile[u];
    const int ntiles = L.nslots / 16;
    const int R = L.nrows;
    const int nbr = (R + CB_BLK - 1) / CB_BLK;
    const bool split = L.slot != 0xffffffffu;
    if (lane < nbr) {   // tiles of each of the unit's block rows, relative to the unit
      const int64_t b = (int64_t)L.brow_lo + lane;
      const int64_t lo = imin64(imax64(a.tile_off[b] - tlo, 0), ntiles);
      const int64_t hi = imin64(imax64(a.tile_off[b + 1] - tlo, lo), ntiles);
      w.tbl[lane] = (int32_t)lo;
      w.tbh[lane] = (int32_t)hi;
    }
    __syncwarp();
    const bool plainx = (L.flags & CB_LUNIT_PLAINX) != 0;
    if (plainx)   // one entry per sub-block (its first column), padded to a multiple of 4
      for (int t = lane; t < ((ntiles + 3) & ~3); t += 32)
        a.lgcols[(size_t)L.gcols + t] = t < ntiles ? 16 * a.tkey[tlo + t] : 0;
    for (int k = lane; k < 16 * ntiles; k += 32) {   // gather list (every slot, in shared memory)
      const int t = k >> 4, c = k & 15;
      int bl = 0;
      while (bl + 1 < nbr && t >= w.tbh[bl]) ++bl;
      const int64_t b = (int64_t)L.brow_lo + bl;
      const int32_t key = a.tkey[tlo + t];
      int32_t cc;
      if (a.agg) {
        const int64_t xb = a.cols_off[b] + 16ll * key + c;
        cc = xb < a.cols_off[b + 1] ? a.rcols[xb] : -1;
      } else {
        const int64_t xb = 16ll * key + c;
        cc = xb < a.n ? (int32_t)xb : -1;
      }
      w.g[k] = cc;
    }
    __syncwarp();
    // per-slot list: uint16 offsets from the smallest column when the columns span fewer
    // than 65,535 values (CB_LUNIT_G16), else the columns themselves
    uint32_t g16 = 0, gbase = 0;
    if (!plainx) {
      int32_t lo = INT32_MAX, hi = -1;
      for (int k = lane; k < 16 * ntiles; k += 32)
        if (w.g[k] >= 0) {
          lo = min(lo, w.g[k]);
          hi = max(hi, w.g[k]);
        }
      for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(kFull, lo, o));
        hi = max(hi, __shfl_xor_sync(kFull, hi, o));
      }
      if (hi >= 0 && (int64_t)hi - lo < 0xffff) {
        g16 = CB_LUNIT_G16;
        gbase = (uint32_t)lo;
        uint16_t* h = reinterpret_cast<uint16_t*>(a.lgcols + L.gcols);
        for (int k = lane; k < 16 * ntiles; k += 32) h[k] = w.g[k] < 0 ? (uint16_t)0xffffu : (uint16_t)(w.g[k] - lo);
      } else {
        for (int k = lane; k < 16 * ntiles; k += 32) a.lgcols[(size_t)L.gcols + k] = w.g[k];
      }
    }
    int carry = 0;
    for (int r0 = 0; r0 < R; r0 += 32) {   // CSR range of every row and their prefix
      const int lr = r0 + lane;
      int cnt = 0, lo = 0;
      if (lr < R) {
        const int64_t r = (int64_t)L.brow_lo * CB_BLK + lr;
        const int64_t ra = a.rp[r], rz = a.rp[r + 1];
        int64_t lo64 = ra, hi64 = rz;
        const int bl = lr >> 4;
        const int s0 = 16 * w.tbl[bl], s1 = 16 * w.tbh[bl];
        if (s1 == s0) {
          hi64 = ra;
        } else if (split) {
          int q = s1 - 1;
          while (q > s0 && w.g[q] < 0) --q;
          lo64 = ra + lower_bound_i32(a.col + ra, (int)(rz - ra), w.g[s0]);
          hi64 = ra + upper_bound_i32(a.col + ra, (int)(rz - ra), w.g[q]);
          if (hi64 < lo64) hi64 = lo64;
        }
        cnt = (int)(hi64 - lo64);
        lo = (int)lo64;
      }
      int inc = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      if (lr < R) {
        w.rlo[lr] = lo;
        w.e[lr + 1] = carry + inc;
      }
      carry += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) w.e[0] = 0;
    __syncwarp();
    const int W = R > 0 ? w.e[R] : 0;
    const int S = L.steps;
    if ((W + 31) / 32 != S) {   // the host's tile counts and the CSR disagree
      if (lane == 0) atomicOr(a.err, kErrUnit);
      __syncwarp();
      continue;
    }
    const int c0 = (lane * W) >> 5, c1 = ((lane + 1) * W) >> 5;
    int lr = 0;
    if (c0 < c1) {   // last row whose first entry is at or before c0
      int lo = 0, hi = R;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.e[mid] <= c0) lo = mid; else hi = mid - 1;
      }
      lr = lo;
    }
    const int vs = a.dtype == CBSPMV_F64 ? 8 : a.dtype == CBSPMV_F32 ? 4 : 2;
    const bool grouped = vs != 8;
    uint64_t wacc = ~0ull;
    bool bad = false;
    for (int st = 0; st < S; ++st) {
      const int k = c0 + st;
      uint64_t v = 0;   // stored bits
      uint32_t word = 0xffffu;
      if (k < c1) {
        while (w.e[lr + 1] <= k) ++lr;
        const int pos = w.rlo[lr] + (k - w.e[lr]);
        const int32_t cc = a.col[pos];
        v = storage_bits(a.val[pos], a.dtype);
        const int bl = lr >> 4;
        int lo = 16 * w.tbl[bl], hi = 16 * w.tbh[bl];
        const int s1 = hi;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((uint32_t)w.g[mid] < (uint32_t)cc) lo = mid + 1; else hi = mid;
        }
        bad |= lo >= s1 || w.g[lo] != cc;
        word = (uint32_t)lo | ((uint32_t)lr << 9);
        if (a.vslot) a.vslot[pos] = L.vals * CB_VLANES + cb_lane_val_index(grouped, (uint32_t)st, (uint32_t)lane, S);
      }
      const size_t vi = (size_t)L.vals * CB_VLANES + cb_lane_val_index(grouped, (uint32_t)st, (uint32_t)lane, S);
      if (vs == 8) reinterpret_cast<uint64_t*>(a.lvals)[vi] = v;
      else if (vs == 4) reinterpret_cast<uint32_t*>(a.lvals)[vi] = (uint32_t)v;
      else reinterpret_cast<uint16_t*>(a.lvals)[vi] = (uint16_t)v;
      const int sh = 16 * (st & 3);
      wacc = (wacc & ~(0xffffull << sh)) | ((uint64_t)word << sh);
      if ((st & 3) == 3 || st == S - 1) {
        a.lwords[(size_t)L.words * CB_VLANES + cb_lane_word_index(grouped, (uint32_t)st, (uint32_t)lane, S)] = wacc;
        wacc = ~0ull;
      }
    }
    if (bad) atomicOr(a.err, kErrUnit);
    int span = 0;   // lanes a row spans (carry resolution by scan above CB_SCAN_SPAN)
    for (int r = lane; r < R; r += 32) {
      const int e0 = w.e[r], e1 = w.e[r + 1];
      if (e1 > e0) span = max(span, (32 * e1 - 1) / W - (32 * (e0 + 1) - 1) / W + 1);
    }
    for (int o = 16; o; o >>= 1) span = max(span, __shfl_xor_sync(kFull, span, o));
    if (lane == 0) {
      a.lunits[u].flags =
          (uint16_t)((L.flags & ~(CB_LUNIT_SCAN | CB_LUNIT_G16)) | (span > CB_SCAN_SPAN ? CB_LUNIT_SCAN : 0) | g16);
      a.lunits[u].gbase = gbase;
    }
    __syncwarp();
  }
}

// rp[min(r0 + j, r1)] for j = 0..16 of every listed block row
__global__ void gather_bounds_kernel(const int64_t* __restrict__ rp, int64_t m, const int32_t* __restrict__ big,
                                     int nbig, int64_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbig * (CB_BLK + 1)) return;
  const int k = i / (CB_BLK + 1), j = i % (CB_BLK + 1);
  const int64_t r0 = (int64_t)big[k] * CB_BLK;
  out[i] = rp[min(r0 + j, m)];
}

}  // namespace

namespace {

// device allocations of one call: temporaries are freed when the call returns, outputs
// only when it fails
struct DevArena {
  DevAllocFn alloc;
  std::vector<void*> temps, outs;
  bool ok_done = false;
  explicit DevArena(DevAllocFn f) : alloc(f) {}
  template <class T>
  cudaError_t get(T** p, size_t count, bool out) {
    *p = nullptr;
    void* q = nullptr;
    const cudaError_t e = alloc(&q, count * sizeof(T) ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    (out ? outs : temps).push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
  ~DevArena() {
    for (void* q : temps) cudaFree(q);
    if (!ok_done)
      for (void* q : outs) cudaFree(q);
  }
};

inline int grid_for(int64_t work, int per_block, int cap) {
  const int64_t g = (work + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace

cbspmv_status_t analyze_device(const cbspmv_csr_t& A, const cbspmv_opts_t& opts, int n_workers, cudaStream_t s,
                               DevAllocFn alloc, Plan* P, DevLanes* out, std::string* msg) {
  const auto t_start = std::chrono::steady_clock::now();
  cbspmv_status_t st = check_opts(opts, n_workers, msg);
  if (st != CBSPMV_OK) return st;
  st = validate_shape(A, msg);
  if (st != CBSPMV_OK) return st;
  if (!uses_lanes(opts)) {
    *msg = "the device analysis builds the lane-stream layout only";
    return CBSPMV_ERR_INVALID;
  }
  *out = DevLanes();
  Plan& p = *P;
  p = Plan();
  p.m = A.m; p.n = A.n; p.nnz = A.nnz;
  p.nbr = (A.m + CB_BLK - 1) / CB_BLK;
  p.value_dtype = opts.value_dtype;
  p.vsize = opts.value_dtype == CBSPMV_F64 ? 8 : opts.value_dtype == CBSPMV_F32 ? 4 : 2;
  p.th0 = opts.th0; p.th1 = opts.th1; p.th2 = opts.th2;
  p.lanes = true;
  const int64_t m = A.m, nbr = p.nbr;
  DevArena ar(alloc);
  cudaError_t e = cudaSuccess;
  auto cuda_fail = [&](cudaError_t r, const char* what) {
    *msg = std::string("device analysis: ") + what + ": " + cudaGetErrorString(r);
    return r == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA;
  };
#define CB_DEV(call, what)                          \
  do {                                              \
    e = (call);                                     \
    if (e != cudaSuccess) return cuda_fail(e, what); \
  } while (0)

  // --- 1. row_ptr ends, then its order, then the columns
  int64_t ends[2] = {0, 0};
  CB_DEV(cudaMemcpyAsync(&ends[0], A.row_ptr, 8, cudaMemcpyDeviceToHost, s), "row_ptr read");
  CB_DEV(cudaMemcpyAsync(&ends[1], A.row_ptr + m, 8, cudaMemcpyDeviceToHost, s), "row_ptr read");
  CB_DEV(cudaStreamSynchronize(s), "row_ptr read");
  if (ends[0] != 0 || ends[1] != A.nnz) {
    *msg = "row_ptr must start at 0 and end at nnz";
    return CBSPMV_ERR_NOT_CANONICAL;
  }
  uint32_t* d_flags = nullptr;   // [0] error flags, [1] large block rows
  int32_t* d_big = nullptr;
  CB_DEV(ar.get(&d_flags, 4, false), "allocation");
  CB_DEV(ar.get(&d_big, (size_t)nbr, false), "allocation");
  CB_DEV(cudaMemsetAsync(d_flags, 0, 16, s), "memset");
  uint32_t flags[2] = {0, 0};
  if (nbr > 0) {
    check_rows_kernel<<<grid_for(nbr, 256, 4096), 256, 0, s>>>(A.row_ptr, m, nbr, d_flags, d_flags + 1, d_big);
    CB_DEV(cudaGetLastError(), "launch");
    CB_DEV(cudaMemcpyAsync(flags, d_flags, 8, cudaMemcpyDeviceToHost, s), "flag read");
    CB_DEV(cudaStreamSynchronize(s), "row check");
    if (flags[0] & kErrRowPtr) {
      *msg = "row_ptr is not non-decreasing";
      return CBSPMV_ERR_NOT_CANONICAL;
    }
    check_cols_kernel<<<grid_for(m, 8, 152 * 32), 256, 0, s>>>(A.row_ptr, A.col_idx, m, A.n, d_flags);
    CB_DEV(cudaGetLastError(), "launch");
  }
  const int nbig = (int)flags[1];

  // --- 2. sorted column multiset of every block row
  int32_t* d_merged = nullptr;
  CB_DEV(ar.get(&d_merged, (size_t)A.nnz, false), "allocation");
  if (nbr > 0) {
    const size_t smem = (size_t)kMergeWarps * 2 * kMergeCap * sizeof(int32_t);
    CB_DEV(cudaFuncSetAttribute(merge_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
           "kernel attribute");
    merge_small_kernel<<<grid_for(nbr, kMergeWarps, 152 * 16), 32 * kMergeWarps, smem, s>>>(A.row_ptr, A.col_idx,
                                                                                             m, nbr, d_merged);
    CB_DEV(cudaGetLastError(), "launch");
  }
  if (nbig > 0) {
    std::vector<int32_t> big(nbig);
    CB_DEV(cudaMemcpyAsync(big.data(), d_big, (size_t)nbig * 4, cudaMemcpyDeviceToHost, s), "list read");
    CB_DEV(cudaStreamSynchronize(s), "list read");
    std::sort(big.begin(), big.end());
    CB_DEV(cudaMemcpyAsync(d_big, big.data(), (size_t)nbig * 4, cudaMemcpyHostToDevice, s), "list write");
    int64_t* d_bnd = nullptr;
    CB_DEV(ar.get(&d_bnd, (size_t)nbig * (CB_BLK + 1), false), "allocation");
    gather_bounds_kernel<<<grid_for((int64_t)nbig * (CB_BLK + 1), 256, 1 << 20), 256, 0, s>>>(A.row_ptr, m, d_big,
                                                                                              nbig, d_bnd);
    CB_DEV(cudaGetLastError(), "launch");
    std::vector<int64_t> bnd((size_t)nbig * (CB_BLK + 1));
    CB_DEV(cudaMemcpyAsync(bnd.data(), d_bnd, bnd.size() * 8, cudaMemcpyDeviceToHost, s), "bounds read");
    CB_DEV(cudaStreamSynchronize(s), "bounds read");
    // chunks of the four merge levels; level L merges runs of 2^L rows
    std::vector<MergeItem> items;
    int level_off[5] = {0, 0, 0, 0, 0};
    for (int L = 0; L < 4; ++L) {
      const int w = 1 << L;
      for (int k = 0; k < nbig; ++k) {
        const int64_t* bk = bnd.data() + (size_t)k * (CB_BLK + 1);
        for (int q = 0; q < CB_BLK; q += 2 * w) {
          const int64_t a0 = bk[q], a1 = bk[std::min(q + w, CB_BLK)], b1 = bk[std::min(q + 2 * w, CB_BLK)];
          for (int64_t d0 = 0; d0 < b1 - a0; d0 += kBigChunk)
            items.push_back(MergeItem{a0, (int32_t)(a1 - a0), (int32_t)(b1 - a1), (int32_t)d0, 0});
        }
      }
      level_off[L + 1] = (int)items.size();
    }
    MergeItem* d_items = nullptr;
    int32_t* d_tmp = nullptr;
    CB_DEV(ar.get(&d_items, items.size(), false), "allocation");
    CB_DEV(ar.get(&d_tmp, (size_t)A.nnz, false), "allocation");
    CB_DEV(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(MergeItem), cudaMemcpyHostToDevice, s),
           "upload");
    // CSR -> tmp -> merged -> tmp -> merged
    const int32_t* src[4] = {A.col_idx, d_tmp, d_merged, d_tmp};
    int32_t* dst[4] = {d_tmp, d_merged, d_tmp, d_merged};
    for (int L = 0; L < 4; ++L) {
      const int n_items = level_off[L + 1] - level_off[L];
      if (n_items == 0) continue;
      merge_big_kernel<<<grid_for(n_items, 1, 152 * 8), kBigThreads, 0, s>>>(d_items + level_off[L], n_items, src[L],
                                                                            dst[L]);
      CB_DEV(cudaGetLastError(), "launch");
    }
    CB_DEV(cudaStreamSynchronize(s), "merge");   // the host vectors above go out of scope
  }

  // --- 3. plain tiles, super-sparse share and distinct columns; aggregation decision
  int32_t *d_nplain = nullptr, *d_ndist = nullptr;
  unsigned long long* d_tot = nullptr;
  CB_DEV(ar.get(&d_nplain, (size_t)nbr, false), "allocation");
  CB_DEV(ar.get(&d_ndist, (size_t)nbr, false), "allocation");
  CB_DEV(ar.get(&d_tot, 2, false), "allocation");
  CB_DEV(cudaMemsetAsync(d_tot, 0, 16, s), "memset");
  std::vector<int32_t> nplain(nbr), ndist(nbr);
  unsigned long long tot[2] = {0, 0};
  if (nbr > 0) {
    tile_count_kernel<<<grid_for(nbr, 8, 152 * 32), 256, 0, s>>>(A.row_ptr, d_merged, m, nbr, opts.th1, d_nplain,
                                                                 d_ndist, d_tot);
    CB_DEV(cudaGetLastError(), "launch");
    CB_DEV(cudaMemcpyAsync(nplain.data(), d_nplain, (size_t)nbr * 4, cudaMemcpyDeviceToHost, s), "count read");
    CB_DEV(cudaMemcpyAsync(ndist.data(), d_ndist, (size_t)nbr * 4, cudaMemcpyDeviceToHost, s), "count read");
  }
  CB_DEV(cudaMemcpyAsync(tot, d_tot, 16, cudaMemcpyDeviceToHost, s), "count read");
  CB_DEV(cudaMemcpyAsync(flags, d_flags, 4, cudaMemcpyDeviceToHost, s), "flag read");
  CB_DEV(cudaStreamSynchronize(s), "tile count");
  if (flags[0] & kErrCols) {
    *msg = "column indices must be strictly increasing within a row and lie in [0, n)";
    return CBSPMV_ERR_NOT_CANONICAL;
  }
  const int64_t plain_tiles = (int64_t)tot[0];
  const double frac = plain_tiles ? (double)tot[1] / (double)plain_tiles : 0.0;
  p.aggregated = opts.col_agg < 0 ? (frac > opts.th0) : (opts.col_agg == 1);
  const bool agg = p.aggregated;
  std::vector<int64_t> tile_off(nbr + 1, 0);
  p.cols_offset.assign(agg ? nbr + 1 : 0, 0);
  for (int64_t b = 0; b < nbr; ++b) {
    tile_off[b + 1] = tile_off[b] + (agg ? (ndist[b] + 15) / 16 : nplain[b]);
    if (agg) p.cols_offset[b + 1] = p.cols_offset[b] + ndist[b];
  }
  const int64_t ntiles = tile_off[nbr];
  if (ntiles >= (1LL << 32)) {
    *msg = "too many tiles";
    return CBSPMV_ERR_UNSUPPORTED;
  }
  p.restore_cols_len = agg ? p.cols_offset[nbr] : 0;

  // --- tiles of every block row (and restore_cols)
  int64_t *d_toff = nullptr, *d_coff = nullptr;
  uint16_t* d_tnnz = nullptr;
  int32_t* d_tkey = nullptr;
  CB_DEV(ar.get(&d_toff, (size_t)nbr + 1, false), "allocation");
  CB_DEV(ar.get(&d_coff, agg ? (size_t)nbr + 1 : 1, false), "allocation");
  CB_DEV(ar.get(&d_tnnz, (size_t)ntiles, false), "allocation");
  CB_DEV(ar.get(&d_tkey, (size_t)ntiles, false), "allocation");
  if (agg) {
    CB_DEV(ar.get(&out->rcols, (size_t)p.restore_cols_len + CB_RC_PAD, true), "allocation");
    CB_DEV(cudaMemsetAsync(out->rcols, 0, ((size_t)p.restore_cols_len + CB_RC_PAD) * 4, s), "memset");
    CB_DEV(cudaMemcpyAsync(d_coff, p.cols_offset.data(), (size_t)(nbr + 1) * 8, cudaMemcpyHostToDevice, s), "upload");
  }
  CB_DEV(cudaMemcpyAsync(d_toff, tile_off.data(), (size_t)(nbr + 1) * 8, cudaMemcpyHostToDevice, s), "upload");
  std::vector<uint16_t> tnnz(ntiles);
  std::vector<int32_t> tkey(ntiles);
  if (nbr > 0) {
    tile_write_kernel<<<grid_for(nbr, 8, 152 * 32), 256, 0, s>>>(A.row_ptr, d_merged, m, nbr, agg ? 1 : 0, d_toff,
                                                                 d_coff, d_tnnz, d_tkey, out->rcols);
    CB_DEV(cudaGetLastError(), "launch");
  }
  if (ntiles > 0) {
    CB_DEV(cudaMemcpyAsync(tnnz.data(), d_tnnz, (size_t)ntiles * 2, cudaMemcpyDeviceToHost, s), "tile read");
    CB_DEV(cudaMemcpyAsync(tkey.data(), d_tkey, (size_t)ntiles * 4, cudaMemcpyDeviceToHost, s), "tile read");
  }
  CB_DEV(cudaStreamSynchronize(s), "tiles");
  try {
    p.tiles.resize(ntiles);
    p.tile_bcol.resize(ntiles);
  } catch (...) {
    *msg = "host allocation failed";
    return CBSPMV_ERR_OOM;
  }
  host_parallel_for(nbr, 1024, [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; ++b)
      for (int64_t t = tile_off[b]; t < tile_off[b + 1]; ++t) {
        CbTile& x = p.tiles[t];
        x.vp16 = 0;
        x.xbase = agg ? (uint32_t)(p.cols_offset[b] + 16 * (int64_t)tkey[t]) : (uint32_t)(16 * (int64_t)tkey[t]);
        x.brow = (uint32_t)b;
        x.nnz = tnnz[t];
        x.fmt = (uint8_t)tile_format(tnnz[t], opts.th1, opts.th2);
        x.pad = 0;
        p.tile_bcol[t] = tkey[t];
      }
  });

  // --- 4. units, load balance and lane offsets on the host; lane programs on the GPU
  cut_units(p, tile_off, opts, n_workers);
  st = check_units(p, msg);
  if (st != CBSPMV_OK) return st;
  std::vector<double> load;
  balance_units(p, opts, n_workers, &load);
  std::vector<uint64_t> voff, woff, goff;
  st = lane_offsets(p, &voff, &woff, &goff, msg);
  if (st != CBSPMV_OK) return st;
  if (opts.keep_value_map && p.n_lane_vals >= (1ull << 32)) {
    *msg = "lane stream too large for a value map";
    return CBSPMV_ERR_UNSUPPORTED;
  }
  const size_t nu = p.units.size();
  std::vector<uint32_t> utile(nu);
  for (size_t i = 0; i < nu; ++i) utile[i] = p.units[i].tile_lo;
  uint32_t* d_utile = nullptr;
  CB_DEV(ar.get(&d_utile, nu, false), "allocation");
  CB_DEV(ar.get(&out->lunits, nu, true), "allocation");
  CB_DEV(ar.get(&out->lvals, p.n_lane_vals * (size_t)p.vsize, true), "allocation");
  CB_DEV(ar.get(&out->lwords, p.n_lane_words, true), "allocation");
  CB_DEV(ar.get(&out->lgcols, p.n_lane_gcols, true), "allocation");
  if (opts.keep_value_map) CB_DEV(ar.get(&out->vslot, (size_t)A.nnz, true), "allocation");
  if (nu > 0) {
    CB_DEV(cudaMemcpyAsync(d_utile, utile.data(), nu * 4, cudaMemcpyHostToDevice, s), "upload");
    CB_DEV(cudaMemcpyAsync(out->lunits, p.lane_units.data(), nu * sizeof(CbLaneUnit), cudaMemcpyHostToDevice, s),
           "upload");
    LaneBuildArgs la{};
    la.rp = A.row_ptr;
    la.col = A.col_idx;
    la.val = A.val;
    la.m = m;
    la.n = A.n;
    la.agg = agg ? 1 : 0;
    la.tile_off = d_toff;
    la.cols_off = d_coff;
    la.tkey = d_tkey;
    la.rcols = out->rcols;
    la.lunits = out->lunits;
    la.utile = d_utile;
    la.nunits = (uint32_t)nu;
    la.dtype = p.value_dtype;
    la.lvals = out->lvals;
    la.lwords = out->lwords;
    la.lgcols = out->lgcols;
    la.vslot = out->vslot;
    la.err = d_flags;
    lane_build_kernel<<<grid_for((int64_t)nu, kBuildWarps, 152 * 8), 32 * kBuildWarps, 0, s>>>(la);
    CB_DEV(cudaGetLastError(), "launch");
    CB_DEV(cudaMemcpyAsync(p.lane_units.data(), out->lunits, nu * sizeof(CbLaneUnit), cudaMemcpyDeviceToHost, s),
           "unit read");
  }
  CB_DEV(cudaMemcpyAsync(flags, d_flags, 4, cudaMemcpyDeviceToHost, s), "flag read");
  CB_DEV(cudaStreamSynchronize(s), "lane build");
  if (flags[0] & kErrUnit) {
    *msg = "internal error: the device lane build disagrees with the tile counts";
    return CBSPMV_ERR_INVALID;
  }
#undef CB_DEV
  out->lvals_count = p.n_lane_vals;
  out->lwords_count = p.n_lane_words;
  out->lgcols_count = p.n_lane_gcols;
  fill_stats(p, plain_tiles, frac, load);
  p.stats.analyzed_on_device = 1;
  ar.ok_done = true;
  p.stats.analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return CBSPMV_OK;
}

}  // namespace cb
