// Run kernel of the blocked SpMV, y = alpha * A * x + beta * y, for sm_103a.
//
// One kernel template serves every value storage type: FP64 values with FP64 x, y and
// accumulation (the paper's setting), and FP32 / BF16 / FP16 values with FP32 x, y and
// accumulation (the mixed-precision storage the paper mentions but does not specify;
// values are widened exactly to FP32 before each FMA).
//
// The paper's kernel (Sec. 3.5, Algorithms 3 and 4) maps one sub-block to one warp,
// preloads x into shared memory (plain tiles) or reads it through restore_cols
// (aggregated tiles), reduces with warp shuffles and adds into y with atomics. On GB300
// the FP64 pipe is the scarce unit (a warp-wide DFMA issues once per 64 cycles on each SM
// sub-partition, and lanes that are masked off cost the same), so this kernel keeps the
// data structure and the per-tile decoding of the paper but reorganises the work:
//
//   * Persistent grid, one CTA per SM; every warp of the CTA is an independent worker
//     with its own shared-memory buffer (as many warps as buffers fit in shared memory).
//     A warp takes the next unit of work of its CTA (a run of consecutive tiles; the
//     CTA's unit list comes from the load balance of Algorithm 2), stages it with two
//     bulk TMA copies (cp.async.bulk: the unit's packed records and its blob of tile
//     records, restore_cols slice and lane schedule) completing on the warp's mbarrier,
//     gathers the unit's x values into its buffer with cp.async (the x preload of
//     Algorithms 3/4, through restore_cols for aggregated tiles) and computes. Warps never
//     wait for one another: the latency of one warp's copies is hidden by the other
//     warps' arithmetic, and the descriptor of a warp's next unit is fetched while it
//     computes the current one.
//   * The analyser's lane schedule cuts the unit's entries, in row-major order, into chunks
//     of at most CB_CHUNK entries of one (tile, row) piece and deals them to the 32 lanes
//     in equal runs. Every lane then runs the same number of steps; a step reads the
//     descriptors of two chunks with one load and issues up to six FMAs into the lane's
//     single row accumulator. No FMA slot is spent on reductions: a row sum is stored when
//     its last chunk is done. For plain units the warp first computes each tile's base
//     addresses from its record (CSR row pointer, COO coordinate bytes of Algorithm 3, the
//     fixed rows of Algorithm 4) and a chunk's 16-bit descriptor names its tile and first
//     entry, whose coordinate bytes give the x columns. Single-entry and consecutive-column
//     units instead carry 32-bit direct descriptors (value offset, tile, first column), and
//     the analyser stores their values in load order, so a chunk needs no tile-base or
//     coordinate load and the lanes of one load read consecutive bytes.
//   * Rows that cross run boundaries are completed by the run holding the row's end
//     (adding the earlier runs' carries in a fixed order); units that cover whole block
//     rows write y directly (no atomics, y read once when beta != 0). Block rows cut into
//     several units store 16 partial sums per part; a second small kernel adds the parts
//     in part order and writes y, so results do not depend on scheduling.
//   * The only wait is a warp's wait for its own bulk copies; it is bounded (clock64
//     budget), and on expiry the kernel records an error code and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "cb_layout.h"
#include "cb_kernels.h"
#include "cb_round.h"

namespace cb {
namespace {

constexpr long long kWaitBudget = 4000000000LL;   // default clock64 budget (~2 s) per wait
constexpr uint32_t kSmemMax = 232448;             // dynamic shared memory per CTA (227 KB)
static_assert(kSmemMax <= (1u << 18), "tile bases are packed as 14 + 18 bits of shared-memory offset");

// Stored value types: V is the storage type, Acc the type of x, y and the accumulators.
template <class V> struct ValT;
// load3: the three consecutive values starting at byte offset va of sm with two aligned
// shared-memory loads (instead of three); it may read up to 4 bytes past the third value.
template <> struct ValT<double> {
  using Acc = double;
  __device__ static __forceinline__ double load(const uint8_t* p) { return *reinterpret_cast<const double*>(p); }
  __device__ static __forceinline__ void load3(const uint8_t* sm, uint32_t va, double& v0, double& v1, double& v2) {
    const bool odd = (va & 8u) != 0;               // va is 8-byte aligned
    const double2 p = *reinterpret_cast<const double2*>(sm + (odd ? va + 8u : va));
    const double q = *reinterpret_cast<const double*>(sm + (odd ? va : va + 16u));
    v0 = odd ? q : p.x;
    v1 = odd ? p.x : p.y;
    v2 = odd ? p.y : q;
  }
};
template <> struct ValT<float> {
  using Acc = float;
  __device__ static __forceinline__ float load(const uint8_t* p) { return *reinterpret_cast<const float*>(p); }
  __device__ static __forceinline__ void load3(const uint8_t* sm, uint32_t va, float& v0, float& v1, float& v2) {
    const uint32_t b = va & ~7u;                   // va is 4-byte aligned
    const float2 p = *reinterpret_cast<const float2*>(sm + b);
    const float2 q = *reinterpret_cast<const float2*>(sm + b + 8u);
    const bool odd = (va & 4u) != 0;
    v0 = odd ? p.y : p.x;
    v1 = odd ? q.x : p.y;
    v2 = odd ? q.y : q.x;
  }
};
// the three 16-bit values starting at byte offset va (2-byte aligned), from two aligned
// 32-bit loads
__device__ __forceinline__ void load3_u16(const uint8_t* sm, uint32_t va, uint32_t& h0, uint32_t& h1, uint32_t& h2) {
  const uint32_t b = va & ~3u;
  const uint32_t w0 = *reinterpret_cast<const uint32_t*>(sm + b);
  const uint32_t w1 = *reinterpret_cast<const uint32_t*>(sm + b + 4u);
  const bool odd = (va & 2u) != 0;
  h0 = odd ? w0 >> 16 : w0 & 0xffffu;
  h1 = odd ? w1 & 0xffffu : w0 >> 16;
  h2 = odd ? w1 >> 16 : w1 & 0xffffu;
}
template <> struct ValT<__nv_bfloat16> {
  using Acc = float;
  __device__ static __forceinline__ float load(const uint8_t* p) {   // exact: bf16 is the top half of fp32
    return __uint_as_float((uint32_t)*reinterpret_cast<const uint16_t*>(p) << 16);
  }
  __device__ static __forceinline__ void load3(const uint8_t* sm, uint32_t va, float& v0, float& v1, float& v2) {
    uint32_t h0, h1, h2;
    load3_u16(sm, va, h0, h1, h2);
    v0 = __uint_as_float(h0 << 16);
    v1 = __uint_as_float(h1 << 16);
    v2 = __uint_as_float(h2 << 16);
  }
};
template <> struct ValT<__half> {
  using Acc = float;
  __device__ static __forceinline__ float load(const uint8_t* p) {   // exact widening
    return __half2float(*reinterpret_cast<const __half*>(p));
  }
  __device__ static __forceinline__ void load3(const uint8_t* sm, uint32_t va, float& v0, float& v1, float& v2) {
    uint32_t h0, h1, h2;
    load3_u16(sm, va, h0, h1, h2);
    v0 = __half2float(__ushort_as_half((unsigned short)h0));
    v1 = __half2float(__ushort_as_half((unsigned short)h1));
    v2 = __half2float(__ushort_as_half((unsigned short)h2));
  }
};

// kK: vectors computed per pass (the product on kK right-hand sides at once).
template <class Acc, int kK>
struct Scratch {
  // per tile, shared-memory offsets of its value base, coordinate base and x row, in one of
  // two forms: q = (value base, coordinate base, x row, 0); w = value base / 16 (bits 0-13)
  // | coordinate base (bits 14-31), the x row following from the tile index
  union {
    uint4 q[CB_T_MAX];
    uint32_t w[CB_T_MAX];
  } tinfo;
  Acc srow[CB_R_MAX * kK];      // row sums, kK per row
  Acc cval[CB_VLANES * kK];     // per-run carry values (short-carry path)
  int32_t crow[CB_VLANES];      // per-run carry row (-1 none, -2 no chunks)
};

__host__ __device__ constexpr uint32_t align128(uint32_t v) { return (v + 127u) & ~127u; }

// Products of one launch: up to kMaxP problems (matrix handle arrays, vectors, scalars)
// passed by value as the kernel parameter. split_base: prefix sums of the problems' split
// block rows (for the combine kernel).
template <int kMaxP>
struct BatchArgs {
  int count;
  uint32_t split_base[kMaxP + 1];   // prefix sums of the problems' split rows with few parts
  uint32_t wide_base[kMaxP + 1];    // prefix sums of their split rows with many parts
  RunArgs p[kMaxP];
};
constexpr int kMaxBatch = 64;

// Per-CTA header: the Dense coordinate bytes, the CTA's unit ticket counter and, for a
// batch, the first unit and the ticket prefix of every problem in this CTA's lists.
struct CtaHeader {
  uint8_t ident[256];           // byte k = (k & 15) << 4: coordinate bytes of a Dense record
  uint64_t never;               // an mbarrier nothing arrives at (the stuck-wait test hook)
  uint32_t ticket;
  uint32_t first[kMaxBatch];    // this CTA's first unit of problem p
  uint32_t pref[kMaxBatch + 1]; // tickets of problems 0..p-1
};
constexpr uint32_t kHeaderBytes = align128(sizeof(CtaHeader));

// Layout of one warp's buffer (byte offsets): the unit descriptor, the unit's packed
// records, its blob (tile records, restore_cols slice, lane schedule), the gathered x
// values (16 per tile), the warp's scratch and its mbarrier.
template <class V, int kK = 1>
struct Geom {
  using Acc = typename ValT<V>::Acc;
  static constexpr uint32_t kBMax = CB_B_MAX_FOR(sizeof(V));
  static constexpr uint32_t kOffUnit = 0;
  static constexpr uint32_t kOffStream = 64;
  static constexpr uint32_t kOffBlob = kOffStream + kBMax;
  static constexpr uint32_t kBlobMax = 16 * CB_T_MAX + 4 * CB_RC_MAX + CB_SCHED_MAX;
  static constexpr uint32_t kOffXs = kOffBlob + kBlobMax;
  static constexpr uint32_t kXRow = 16u * (uint32_t)sizeof(Acc) * kK;   // bytes of a tile's x values
  static constexpr uint32_t kOffScratch = align128(kOffXs + CB_T_MAX * kXRow);
  static constexpr uint32_t kOffBar = kOffScratch + (((uint32_t)sizeof(Scratch<Acc, kK>) + 15u) & ~15u);
  static constexpr uint32_t kWarpBytes = align128(kOffBar + 16);   // two mbarriers: blob, records
  static constexpr uint32_t kFit = (kSmemMax - kHeaderBytes) / kWarpBytes;
  static constexpr int kWarps = kFit > 32 ? 32 : (int)kFit;
  static constexpr uint32_t kSmem = kHeaderBytes + kWarps * kWarpBytes;
  static_assert(kWarps >= 4, "warp buffers too large");
  static_assert(kOffStream % 16 == 0 && kOffBlob % 16 == 0 && kOffXs % 16 == 0 && kBlobMax % 16 == 0,
                "bulk copy destinations must be 16-byte aligned");
};
static_assert(sizeof(CbUnit) == 64, "unit descriptor slot");
static_assert(CB_T_MAX <= 32 && (CB_T_MAX * 16) % 32 == 0, "tile count per unit");

// ---- PTX helpers (mbarrier, bulk copy, cp.async) --------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the budget (clock64 cycles) ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget = kWaitBudget) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// cp.async of one x element (8 or 4 bytes); src_bytes = 0 writes zeros
template <int kBytes>
__device__ __forceinline__ void cp_async_elem(uint32_t dst_smem, const void* src, uint32_t src_bytes) {
  static_assert(kBytes == 8 || kBytes == 4, "x element size");
  if constexpr (kBytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst_smem), "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst_smem), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t align16u(uint32_t v) { return (v + 15u) & ~15u; }

__device__ void set_error(const RunArgs& a, uint32_t code) { atomicOr(a.err, code); }

// ---- staging of one unit by its warp ---------------------------------------------------
__device__ __forceinline__ uint32_t load_desc_word(const CbUnit* units, uint32_t k, uint32_t nu, int lane) {
  return (k < nu && lane < 16) ? __ldg(reinterpret_cast<const uint32_t*>(units + k) + lane) : 0u;
}

// Starts gathering the unit's x values into the warp's buffer: 16 per tile (column c of
// tile t at index 16 t + c), x[restore_cols[xbase + c]] when aggregated, x[xbase + c]
// otherwise; columns outside [0, n) (padding of the last block column) read as zero. The
// cp.async copies are waited for by consume_unit after its set-up.
template <class V, int kK>
__device__ __forceinline__ void gather_x(const RunArgs& a, const uint8_t* W, uint32_t w_smem, int lane) {
  using G = Geom<V, kK>;
  using Acc = typename G::Acc;
  constexpr int kPerLane = CB_T_MAX * 16 / 32;
  constexpr uint32_t kXs = sizeof(Acc);
  const Acc* x = static_cast<const Acc*>(a.x);
  const CbUnit& u = *reinterpret_cast<const CbUnit*>(W + G::kOffUnit);
  const CbTile* tiles = reinterpret_cast<const CbTile*>(W + G::kOffBlob);
  const int32_t* rcols = reinterpret_cast<const int32_t*>(W + G::kOffBlob + 16u * u.ntiles);
  const uint32_t nx = 16u * u.ntiles, rc_lo = u.rc_lo;
  int64_t col[kPerLane];
#pragma unroll
  for (int k = 0; k < kPerLane; ++k) {
    const uint32_t idx = (uint32_t)lane + 32u * k;
    col[k] = -1;
    if (idx < nx) {
      const uint32_t xb = tiles[idx >> 4].xbase;
      col[k] = a.aggregated ? (int64_t)rcols[xb - rc_lo + (idx & 15u)] : (int64_t)xb + (idx & 15u);
    }
  }
#pragma unroll
  for (int k = 0; k < kPerLane; ++k) {
    const uint32_t idx = (uint32_t)lane + 32u * k;
    if (idx < nx) {
      const bool valid = col[k] >= 0 && col[k] < a.n;
#pragma unroll
      for (int j = 0; j < kK; ++j)      // the kK vectors' values of one column side by side
        cp_async_elem<kXs>(w_smem + G::kOffXs + kXs * (idx * kK + j), x + (valid ? col[k] + j * a.ldx : 0),
                           valid ? kXs : 0u);
    }
  }
  // the copies complete while the unit's set-up runs; consume_unit waits for them
}

// ---- a unit's rows ----------------------------------------------------------------------
// acc + v * x when p holds, acc otherwise (a predicated FP64 FMA, no branch).
__device__ __forceinline__ double pfma(bool p, double v, double x, double acc) {
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q fma.rn.f64 %0, %1, %2, %0;\n\t}"
      : "+d"(acc)
      : "d"(v), "d"(x), "r"((uint32_t)p));
  return acc;
}
__device__ __forceinline__ float pfma(bool p, float v, float x, float acc) {
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q fma.rn.f32 %0, %1, %2, %0;\n\t}"
      : "+f"(acc)
      : "f"(v), "f"(x), "r"((uint32_t)p));
  return acc;
}

// kK consecutive Acc values at byte offset off of shared memory (aligned to their size).
template <class Acc, int kK>
__device__ __forceinline__ void load_xk(const uint8_t* sm, uint32_t off, Acc (&x)[kK]) {
  if constexpr (kK * sizeof(Acc) >= 16) {
#pragma unroll
    for (int q = 0; q < (int)(kK * sizeof(Acc) / 16); ++q) {
      const uint4 w = *reinterpret_cast<const uint4*>(sm + off + 16u * q);
      constexpr int per = 16 / (int)sizeof(Acc);
      const Acc* p = reinterpret_cast<const Acc*>(&w);
#pragma unroll
      for (int e = 0; e < per; ++e) x[q * per + e] = p[e];
    }
  } else if constexpr (kK * sizeof(Acc) == 8 && kK == 2) {
    const float2 w = *reinterpret_cast<const float2*>(sm + off);
    x[0] = w.x;
    x[1] = w.y;
  } else {
    x[0] = *reinterpret_cast<const Acc*>(sm + off);
  }
}

// sm: base of the CTA's shared memory; so: offset of the unit's buffer in it. Computes the
// unit's rows for kK vectors (x values of column c of tile t at x-row t, slot c * kK + j).
// kC: entries per chunk of the unit's schedule, CB_CHUNK or 1 (CB_MODE_ENTRY). kX = 1: the
// unit's chunks cover consecutive columns (CB_MODE_XSEQ; single vector), so the chunk's x
// values are contiguous in the tile's x row and are read like its values.
// bar_s / phase: the mbarrier phase on which the unit's records land (waited for after the
// set-up). Returns false if that bounded wait gave up (nothing is written then).
template <class V, int kK, int kC, int kX, int kD>
__device__ bool consume_unit(const RunArgs& a, uint8_t* sm, uint32_t so, uint32_t ident_off,
                             Scratch<typename ValT<V>::Acc, kK>& sc, int lane, uint64_t* bar_s,
                             uint32_t phase) {
  static_assert(kC == CB_CHUNK || kC == 1, "chunk size");
  static_assert(kX == 0 || (kC == CB_CHUNK && (kK == 1 || kD == 1)),
                "contiguous x chunks: single vector unless the descriptors are direct");
  static_assert(kD == 0 || kC == 1 || kX == 1, "direct descriptors: single entries or consecutive columns");
  using Acc = typename ValT<V>::Acc;
  using G = Geom<V, kK>;
  constexpr uint32_t kOffUnit = G::kOffUnit, kOffStream = G::kOffStream, kOffBlob = G::kOffBlob,
                     kOffXs = G::kOffXs;
  constexpr uint32_t kVs = sizeof(V), kXs = sizeof(Acc);
  // byte offset of column c's x values in the tile's x row for a coordinate byte b
  // (c = b >> 4): c * kXs * kK
  constexpr uint32_t kXStride = kXs * kK;
  uint8_t* S = sm + so;
  const CbUnit& u = *reinterpret_cast<const CbUnit*>(S + kOffUnit);
  const uint32_t T = u.ntiles;
  const uint32_t byte_lo = u.byte_lo16 * 16u;
  const int64_t row0 = (int64_t)u.brow_lo * CB_BLK;
  const int64_t rows_left = a.m - row0;
  const int64_t rows_unit = (int64_t)CB_BLK * u.nbr;
  const uint32_t R = (uint32_t)(rows_unit < rows_left ? rows_unit : rows_left);
  const CbTile* tiles = reinterpret_cast<const CbTile*>(S + kOffBlob);
  const bool scan_carries = (u.mode & CB_MODE_SCAN) != 0;
  // Tile bases as one 32-bit word (one conflict-free load per chunk when a warp's lanes read
  // many tiles), except for FP64 consecutive-column units: their lanes mostly share a few
  // tiles, the 16-byte load is then a broadcast, and the word's decode on the load chain
  // measured slower.
  constexpr bool kPacked = !(sizeof(V) == 8 && kX == 1);

  // 1. per-tile bases (lane = tile; not needed with direct descriptors) and zeroed row sums
  if (!kD && (uint32_t)lane < T) {
    const CbTile rec = tiles[lane];
    const uint32_t soff = so + kOffStream + rec.vp16 * 16u - byte_lo;
    uint32_t vb, cb;
    if (rec.fmt == CB_FMT_CSR) {
      vb = soff + align16u(17u + rec.nnz);
      cb = soff + 17u;
    } else if (rec.fmt == CB_FMT_DENSE) {
      vb = soff + 32u;
      cb = ident_off;
    } else {
      vb = soff + align16u(rec.nnz);
      cb = soff;
    }
    if constexpr (kPacked) sc.tinfo.w[lane] = (vb >> 4) | (cb << 14);
    else sc.tinfo.q[lane] = make_uint4(vb, cb, so + kOffXs + G::kXRow * lane, 0u);
  }
  for (uint32_t r = lane; r < R * kK; r += 32) sc.srow[r] = Acc(0);
  if (!__all_sync(0xffffffffu, mbar_wait(bar_s, phase, a.wait_budget))) return false;   // the records
  cp_async_wait_all();     // this lane's x copies (issued by gather_x before the set-up)
  __syncwarp();

  // 2. one run per lane: a sequence of chunks of up to three entries, accumulated in one
  //    chain per vector. A second chain would hide no latency (a warp-wide FP64 FMA holds
  //    its sub-partition's pipe for 64 cycles, longer than the FMA's latency) and would
  //    cost an FP64 add at every row end.
  const uint8_t* sched = S + kOffBlob + 16u * T + 4u * u.rc_n;
  const uint16_t* hdr = reinterpret_cast<const uint16_t*>(sched);
  const uint8_t* nxt = sched + 2 * CB_VLANES;
  // descriptor pairs: two 16-bit descriptors in one 32-bit word, or (direct) two 32-bit
  // descriptors in one 64-bit word
  const uint32_t* desc = reinterpret_cast<const uint32_t*>(sched + CB_SCHED_HDR(R));
  const uint2* desc2 = reinterpret_cast<const uint2*>(sched + CB_SCHED_HDR(R));
  const uint32_t h = hdr[lane];
  const uint32_t nch = h >> 9;
  const uint32_t nmax = __reduce_max_sync(0xffffffffu, nch);
  const uint32_t steps = (nmax + 1) / 2;
  uint32_t row = h & 0xffu;
  const bool hs = (h >> 8) & 1u;
  bool first = true, open = false;
  int32_t own_row = -1;
  Acc own_val[kK], acc[kK];
#pragma unroll
  for (int j = 0; j < kK; ++j) own_val[j] = acc[j] = Acc(0);
  // Software pipeline: the operands of step i + 1 are loaded before the FMAs of step i.
  // Loads are unconditional (a chunk shorter than three entries reads at most two entries,
  // plus up to 4 value bytes and 5 coordinate bytes of alignment slack, past its piece;
  // column nibbles stay inside the tile's x row, so every address stays in the warp's
  // buffer or the CTA header); the FMA slots beyond the chunk's length are predicated off.
  uint32_t dA = 0, dB = 0;
  Acc vA0 = 0, vA1 = 0, vA2 = 0, vB0 = 0, vB1 = 0, vB2 = 0;
  Acc xA0[kK], xA1[kK], xA2[kK], xB0[kK], xB1[kK], xB2[kK];
#pragma unroll
  for (int j = 0; j < kK; ++j) xA0[j] = xA1[j] = xA2[j] = xB0[j] = xB1[j] = xB2[j] = Acc(0);
  // (b >> 4) * stride for b < 256 and a power-of-two stride, in two operations
  constexpr uint32_t kXLog = kXStride == 4 ? 2 : kXStride == 8 ? 3 : kXStride == 16 ? 4 : 5;
  static_assert((1u << kXLog) == kXStride, "x stride must be 4, 8, 16 or 32 bytes");
#define CB_XOFF(b_) (kXLog <= 4 ? (((b_) >> (4 - (kXLog <= 4 ? kXLog : 4))) & (15u << kXLog)) \
                                : (((b_) & 0xF0u) << (kXLog > 4 ? kXLog - 4 : 0)))
#define CB_LOAD_CHUNK(d, v0, v1, v2, x0, x1, x2)                                   \
  if constexpr (kD) {                                                              \
    const uint32_t va_ = vrec0 + (((d) & 0xfffu) << 1);                            \
    const uint32_t xa_ = xrow0 + G::kXRow * (((d) >> 12) & 31u) + kXStride * (((d) >> 17) & 15u); \
    if constexpr (kC == 1) {                                                       \
      v0 = ValT<V>::load(sm + va_);                                                \
      load_xk<Acc, kK>(sm, xa_, x0);                                               \
    } else {                                                                       \
      ValT<V>::load3(sm, va_, v0, v1, v2);                                         \
      if constexpr (kK == 1) {                                                     \
        ValT<Acc>::load3(sm, xa_, x0[0], x1[0], x2[0]);                            \
      } else {                                                                     \
        load_xk<Acc, kK>(sm, xa_, x0);                                             \
        load_xk<Acc, kK>(sm, xa_ + kXStride, x1);                                  \
        load_xk<Acc, kK>(sm, xa_ + 2u * kXStride, x2);                             \
      }                                                                            \
    }                                                                              \
  } else {                                                                         \
    const uint32_t o_ = ((d) >> 5) & 255u;                                         \
    uint32_t va_, ca_, xr_;                                                        \
    if constexpr (kPacked) {                                                       \
      const uint32_t ti_ = sc.tinfo.w[(d) & 31u];                                  \
      va_ = ((ti_ & 0x3fffu) << 4) + kVs * o_;                                     \
      ca_ = (ti_ >> 14) + o_;                                                      \
      xr_ = xrow0 + G::kXRow * ((d) & 31u);                                        \
    } else {                                                                       \
      const uint4 ti_ = sc.tinfo.q[(d) & 31u];                                     \
      va_ = ti_.x + kVs * o_;                                                      \
      ca_ = ti_.y + o_;                                                            \
      xr_ = ti_.z;                                                                 \
    }                                                                              \
    if constexpr (kC == 1) {                                                       \
      v0 = ValT<V>::load(sm + va_);                                                \
      load_xk<Acc, kK>(sm, xr_ + CB_XOFF((uint32_t)sm[ca_]), x0);                  \
    } else if constexpr (kX == 1) {                                                \
      ValT<V>::load3(sm, va_, v0, v1, v2);                                         \
      ValT<Acc>::load3(sm, xr_ + CB_XOFF((uint32_t)sm[ca_]), x0[0], x1[0], x2[0]); \
    } else {                                                                       \
      const uint32_t cw_ = ca_ & ~3u;                                              \
      const uint32_t cb_ = __funnelshift_r(*reinterpret_cast<const uint32_t*>(sm + cw_), \
                                           *reinterpret_cast<const uint32_t*>(sm + cw_ + 4u), \
                                           8u * (ca_ & 3u));                       \
      const uint32_t b0_ = cb_ & 0xffu, b1_ = (cb_ >> 8) & 0xffu, b2_ = (cb_ >> 16) & 0xffu; \
      ValT<V>::load3(sm, va_, v0, v1, v2);                                         \
      load_xk<Acc, kK>(sm, xr_ + CB_XOFF(b0_), x0);                                \
      load_xk<Acc, kK>(sm, xr_ + CB_XOFF(b1_), x1);                                \
      load_xk<Acc, kK>(sm, xr_ + CB_XOFF(b2_), x2);                                \
    }                                                                              \
  }
  const uint32_t xrow0 = so + kOffXs;      // x row of tile 0
  const uint32_t vrec0 = so + kOffStream;  // the unit's first stream byte
  // the pair of descriptors of step i
  auto desc_pair = [&](uint32_t i, uint32_t& da, uint32_t& db) {
    if constexpr (kD) {
      const uint2 dd = desc2[i * CB_VLANES + lane];
      da = dd.x;
      db = dd.y;
    } else {
      const uint32_t dd = desc[i * CB_VLANES + lane];
      da = dd & 0xffffu;
      db = dd >> 16;
    }
  };
  // length (0..3) and row-end flag of a descriptor
  constexpr uint32_t kLenShift = kD ? 21 : 13, kEndBit = kD ? (1u << 23) : 0x8000u;
  if (steps) {
    desc_pair(0, dA, dB);
    CB_LOAD_CHUNK(dA, vA0, vA1, vA2, xA0, xA1, xA2);
    CB_LOAD_CHUNK(dB, vB0, vB1, vB2, xB0, xB1, xB2);
  }
  for (uint32_t i = 0; i < steps; ++i) {
    uint32_t dA_n, dB_n;
    desc_pair(i + 1 < steps ? i + 1 : i, dA_n, dB_n);
    Acc nvA0, nvA1 = Acc(0), nvA2 = Acc(0), nvB0, nvB1 = Acc(0), nvB2 = Acc(0);
    Acc nxA0[kK], nxA1[kK], nxA2[kK], nxB0[kK], nxB1[kK], nxB2[kK];
    CB_LOAD_CHUNK(dA_n, nvA0, nvA1, nvA2, nxA0, nxA1, nxA2);
    CB_LOAD_CHUNK(dB_n, nvB0, nvB1, nvB2, nxB0, nxB1, nxB2);
    const uint32_t lA = (dA >> kLenShift) & 3u, lB = (dB >> kLenShift) & 3u;
    const bool eA = (dA & kEndBit) != 0, eB = (dB & kEndBit) != 0;
    // chunk A, then chunk B, into the chain; when chunk A ends its row, its sum is kept
    // aside and chunk B starts a new row from zero
    Acc sA[kK];
#pragma unroll
    for (int j = 0; j < kK; ++j) {
      Acc c = pfma(lA > 0, vA0, xA0[j], acc[j]);
      if constexpr (kC > 1) {
        c = pfma(lA > 1, vA1, xA1[j], c);
        c = pfma(lA > 2, vA2, xA2[j], c);
      }
      sA[j] = c;
      c = eA ? Acc(0) : c;
      c = pfma(lB > 0, vB0, xB0[j], c);
      if constexpr (kC > 1) {
        c = pfma(lB > 1, vB1, xB1[j], c);
        c = pfma(lB > 2, vB2, xB2[j], c);
      }
      acc[j] = c;
    }
    if (lA | lB) open = true;
    if (eA) {                              // chunk A ends its row
      const bool own = first && hs;
      if (own) own_row = (int32_t)row;
#pragma unroll
      for (int j = 0; j < kK; ++j) {
        if (own) own_val[j] = sA[j];
        else sc.srow[row * kK + j] = sA[j];
      }
      first = false;
      open = lB != 0;
      row = nxt[row];
    }
    if (eB) {                              // chunk B ends its row
      const bool own = first && hs;
      if (own) own_row = (int32_t)row;
#pragma unroll
      for (int j = 0; j < kK; ++j) {
        if (own) own_val[j] = acc[j];
        else sc.srow[row * kK + j] = acc[j];
        acc[j] = Acc(0);
      }
      first = false;
      open = false;
      row = nxt[row];
    }
    dA = dA_n;
    dB = dB_n;
    vA0 = nvA0; vA1 = nvA1; vA2 = nvA2;
    vB0 = nvB0; vB1 = nvB1; vB2 = nvB2;
#pragma unroll
    for (int j = 0; j < kK; ++j) {
      xA0[j] = nxA0[j]; xA1[j] = nxA1[j]; xA2[j] = nxA2[j];
      xB0[j] = nxB0[j]; xB1[j] = nxB1[j]; xB2[j] = nxB2[j];
    }
  }
#undef CB_LOAD_CHUNK
#undef CB_XOFF
  // Rows crossing runs: a lane whose run ends inside a row carries that row's partial sum;
  // the lane where the row ends (own_row) adds the carries of the lanes before it, in a
  // fixed order. Rows spanning a few lanes: the owner walks back over them (skipping lanes
  // without chunks). Units where a row spans more than CB_SCAN_SPAN lanes (analyser flag
  // CB_MODE_SCAN): a segmented inclusive scan over lanes (Hillis-Steele, 5 steps); lanes
  // without chunks take the key of the last lane with chunks before them and carry zero.
  if (!scan_carries) {
    sc.crow[lane] = nch == 0 ? -2 : (open ? (int32_t)row : -1);
#pragma unroll
    for (int j = 0; j < kK; ++j) sc.cval[lane * kK + j] = open ? acc[j] : Acc(0);
    __syncwarp();
    if (own_row >= 0) {
      Acc sum[kK];
#pragma unroll
      for (int j = 0; j < kK; ++j) sum[j] = own_val[j];
      for (int l = (int)lane - 1; l >= 0; --l) {
        const int32_t cr = sc.crow[l];
        if (cr == -2) continue;
        if (cr != own_row) break;
#pragma unroll
        for (int j = 0; j < kK; ++j) sum[j] += sc.cval[l * kK + j];
      }
#pragma unroll
      for (int j = 0; j < kK; ++j) sc.srow[own_row * kK + j] = sum[j];
    }
  } else {
    constexpr uint32_t kFull = 0xffffffffu;
    const int32_t key0 = nch == 0 ? -2 : (open ? (int32_t)row : -1);
    int last = nch == 0 ? -1 : lane;               // last lane with chunks up to this one
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(kFull, last, d);
      if (lane >= d && o > last) last = o;
    }
    const int32_t key = __shfl_sync(kFull, key0, last < 0 ? lane : last);
    Acc cv[kK];
#pragma unroll
    for (int j = 0; j < kK; ++j) cv[j] = open ? acc[j] : Acc(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t ko = __shfl_up_sync(kFull, key, d);
      const bool take = lane >= d && ko == key;
#pragma unroll
      for (int j = 0; j < kK; ++j) {
        const Acc vo = __shfl_up_sync(kFull, cv[j], d);
        if (take) cv[j] += vo;
      }
    }
    const int32_t kprev = __shfl_up_sync(kFull, key, 1);
#pragma unroll
    for (int j = 0; j < kK; ++j) {
      const Acc prev = __shfl_up_sync(kFull, cv[j], 1);
      if (own_row >= 0) sc.srow[own_row * kK + j] = own_val[j] + (kprev == own_row ? prev : Acc(0));
    }
  }
  __syncwarp();

  // 3. outputs (alpha and beta in the accumulation type)
  const Acc alpha = (Acc)a.alpha, beta = (Acc)a.beta;
  Acc* y = static_cast<Acc*>(a.y);
  if (u.split < 0) {
    for (uint32_t r = lane; r < R; r += 32) {
      const int64_t gr = row0 + r;
#pragma unroll
      for (int j = 0; j < kK; ++j) {
        Acc* yj = y + (int64_t)j * a.ldy;
        Acc v = sc.srow[r * kK + j];
        if (!a.alpha_one) v = alpha * v;
        if (a.beta_nonzero) v = fma(beta, yj[gr], v);
        yj[gr] = v;
      }
    }
  } else {
    // part of a block row cut into several units: 16 x kK partial sums, added by
    // combine_kernel
    Acc* partial = static_cast<Acc*>(a.partial);
    if (lane < 16) {
#pragma unroll
      for (int j = 0; j < kK; ++j)
        partial[((size_t)u.slot * 16 + lane) * kK + j] = (uint32_t)lane < R ? sc.srow[lane * kK + j] : Acc(0);
    }
  }
  return true;
}

template <class V, int kMaxP, int kK>
__global__ void __launch_bounds__(32 * Geom<V, kK>::kWarps, 1) spmv_kernel(const __grid_constant__ BatchArgs<kMaxP> b) {
  using G = Geom<V, kK>;
  using Acc = typename G::Acc;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  CtaHeader& hd = *reinterpret_cast<CtaHeader*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t wo = kHeaderBytes + (uint32_t)warp * G::kWarpBytes;   // this warp's buffer
  uint8_t* W = smem_raw + wo;
  const uint32_t w_smem = smem_u32(W);
  uint64_t* bar = reinterpret_cast<uint64_t*>(W + G::kOffBar);   // the unit's blob landed
  uint64_t* bar_s = bar + 1;                                      // the unit's records landed
  Scratch<Acc, kK>& sc = *reinterpret_cast<Scratch<Acc, kK>*>(W + G::kOffScratch);
  // this CTA's unit lists of the batch's problems (stored contiguously per CTA), one after
  // another in ticket order
  const int P = b.count;
  if ((int)threadIdx.x < P) {
    const RunArgs& a = b.p[threadIdx.x];
    const uint32_t w0 = a.worker_off[blockIdx.x];
    hd.first[threadIdx.x] = w0;
    hd.pref[threadIdx.x + 1] = a.worker_off[blockIdx.x + 1] - w0;
  }
  if (threadIdx.x == 0) {
    hd.ticket = 0;
    mbar_init(&hd.never, 1);
  }
  for (uint32_t i = threadIdx.x; i < 256u; i += blockDim.x) hd.ident[i] = (uint8_t)((i & 15u) << 4);
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init(bar_s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    hd.pref[0] = 0;
    for (int q = 0; q < P; ++q) hd.pref[q + 1] += hd.pref[q];
  }
  __syncthreads();
  const uint32_t total = hd.pref[P];
  const uint32_t ident_off = (uint32_t)(hd.ident - smem_raw);
  auto grab = [&]() -> uint32_t {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&hd.ticket, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
  };
  // problem of ticket t (t < total): the last q with pref[q] <= t
  auto problem_of = [&](uint32_t t) -> int {
    if (kMaxP == 1) return 0;
    int lo = 0, hi = P - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (hd.pref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  auto desc_word = [&](uint32_t t) -> uint32_t {
    if (t >= total) return 0u;
    const int q = problem_of(t);
    return load_desc_word(b.p[q].units + hd.first[q], t - hd.pref[q], 0xffffffffu, lane);
  };
  uint32_t phase = 0;
  uint32_t j = grab();
  uint32_t dw = desc_word(j);
  while (j < total) {
    const RunArgs& a = b.p[problem_of(j)];
    if (lane < 16) reinterpret_cast<uint32_t*>(W + G::kOffUnit)[lane] = dw;
    __syncwarp();
    if (lane == 0) {
      // the buffer was last read and written through the generic proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const CbUnit& u = *reinterpret_cast<const CbUnit*>(W + G::kOffUnit);
      mbar_arrive_expect_tx(bar, u.blob_bytes);
      if (u.blob_bytes) bulk_g2s(W + G::kOffBlob, a.blob + (size_t)u.blob16 * 16, u.blob_bytes, bar);
      mbar_arrive_expect_tx(bar_s, u.nbytes);
      if (u.nbytes) bulk_g2s(W + G::kOffStream, a.stream + (size_t)u.byte_lo16 * 16, u.nbytes, bar_s);
    }
    // the next unit's descriptor is fetched while this one is staged and computed
    const uint32_t jn = grab();
    const uint32_t dwn = desc_word(jn);
    // the blob (tile records, restore_cols slice, schedule) is enough to start the x
    // gather and the unit's set-up; the records are waited for just before the walk
    // (test hook: the first wait of a stuck-wait run is on a barrier nothing arrives at)
    bool ok = __all_sync(0xffffffffu, mbar_wait(a.stuck_wait ? &hd.never : bar, phase, a.wait_budget));
    if (ok) {
      gather_x<V, kK>(a, W, w_smem, lane);
      __syncwarp();
      const uint32_t mode = reinterpret_cast<const CbUnit*>(W + G::kOffUnit)->mode;
      if (mode & CB_MODE_DIRECT) {
        if (mode & CB_MODE_ENTRY)
          ok = consume_unit<V, kK, 1, 0, 1>(a, smem_raw, wo, ident_off, sc, lane, bar_s, phase);
        else
          ok = consume_unit<V, kK, CB_CHUNK, 1, 1>(a, smem_raw, wo, ident_off, sc, lane, bar_s, phase);
      } else if (mode & CB_MODE_ENTRY) {
        ok = consume_unit<V, kK, 1, 0, 0>(a, smem_raw, wo, ident_off, sc, lane, bar_s, phase);
      } else if (kK == 1 && (mode & CB_MODE_XSEQ)) {
        ok = consume_unit<V, kK, CB_CHUNK, (kK == 1 ? 1 : 0), 0>(a, smem_raw, wo, ident_off, sc, lane, bar_s,
                                                                phase);
      } else {
        ok = consume_unit<V, kK, CB_CHUNK, 0, 0>(a, smem_raw, wo, ident_off, sc, lane, bar_s, phase);
      }
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) set_error(a, 2u);
      // copies may still land in the buffer: give them a second bounded wait with the full
      // budget (whatever the run's budget), then stop
      mbar_wait(bar, phase);
      mbar_wait(bar_s, phase);
      cp_async_wait_all();
      break;
    }
    phase ^= 1u;
    j = jn;
    dw = dwn;
  }
}

// Adds the parts of every block row cut into several units, in part order, and writes y.
template <class Acc, int kMaxP, int kK>
__device__ __forceinline__ void combine_narrow(const BatchArgs<kMaxP>& b, uint32_t blk) {
  const uint32_t g = blk * 256u + threadIdx.x;
  const uint32_t srg = g >> 4, r = g & 15u;
  if (srg >= b.split_base[b.count]) return;
  int q = 0;
  if (kMaxP > 1) {
    int lo = 0, hi = b.count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.split_base[mid] <= srg) lo = mid; else hi = mid - 1;
    }
    q = lo;
  }
  const RunArgs& a = b.p[q];
  const CbSplitRow s = a.split_rows[srg - b.split_base[q]];   // rows with few parts come first
  if (r >= s.rows) return;
  const int64_t gr = (int64_t)s.brow * CB_BLK + r;
#pragma unroll
  for (int j = 0; j < kK; ++j) {
    const Acc* p = static_cast<const Acc*>(a.partial) + ((size_t)s.slot0 * 16 + r) * kK + j;
    constexpr size_t kPart = 16 * kK;   // distance between parts
    // Up to four parts: added in part order, nparts - 1 adds (an FP64 add holds the FP64
    // pipe as long as an FMA does, so none is spent on adding zeros). More parts:
    // parts k = q (mod 4) into four chains started from the first four parts, then a fixed
    // tree.
    Acc sum;
    if (s.nparts <= 4) {
      sum = p[0];
      for (uint32_t k = 1; k < s.nparts; ++k) sum += p[k * kPart];
    } else {
      Acc t[4] = {p[0], p[kPart], p[2 * kPart], p[3 * kPart]};
      uint32_t k = 4;
      for (; k + 4 <= s.nparts; k += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] += p[(size_t)(k + q) * kPart];
      }
      if (k < s.nparts) t[0] += p[(size_t)k * kPart];
      if (k + 1 < s.nparts) t[1] += p[(size_t)(k + 1) * kPart];
      if (k + 2 < s.nparts) t[2] += p[(size_t)(k + 2) * kPart];
      sum = (t[0] + t[1]) + (t[2] + t[3]);
    }
    Acc* y = static_cast<Acc*>(a.y) + (int64_t)j * a.ldy;
    Acc v = a.alpha_one ? sum : (Acc)a.alpha * sum;
    if (a.beta_nonzero) v = fma((Acc)a.beta, y[gr], v);
    y[gr] = v;
  }
}

// Split rows with many parts (the last n_split_wide of each problem): one block of 256
// threads per row, 16 lanes per row of the block row; lane l adds parts l, l + 16, ... in
// four independent sums, then the 16 lanes' sums are added by a fixed shuffle tree. Rows of
// power-law matrices can have hundreds of parts: with one thread per row, every iteration
// would wait a full memory latency.
template <class Acc, int kMaxP, int kK>
__device__ __forceinline__ void combine_wide(const BatchArgs<kMaxP>& b, uint32_t blk) {
  const uint32_t srg = blk;
  const uint32_t r = threadIdx.x >> 4, lane = threadIdx.x & 15u;
  int q = 0;
  if (kMaxP > 1) {
    int lo = 0, hi = b.count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.wide_base[mid] <= srg) lo = mid; else hi = mid - 1;
    }
    q = lo;
  }
  const RunArgs& a = b.p[q];
  const CbSplitRow s = a.split_rows[a.n_split_rows - a.n_split_wide + (srg - b.wide_base[q])];
  const int64_t gr = (int64_t)s.brow * CB_BLK + r;
#pragma unroll
  for (int j = 0; j < kK; ++j) {
    const Acc* p = static_cast<const Acc*>(a.partial) + ((size_t)s.slot0 * 16 + r) * kK + j;
    Acc t[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
    uint32_t k = lane;
    for (; k + 48 < s.nparts; k += 64) {
#pragma unroll
      for (int u = 0; u < 4; ++u) t[u] += p[(size_t)(k + 16 * u) * 16 * kK];
    }
    for (int u = 0; k < s.nparts; k += 16, ++u) {
      if (u == 0) t[0] += p[(size_t)k * 16 * kK];
      else if (u == 1) t[1] += p[(size_t)k * 16 * kK];
      else t[2] += p[(size_t)k * 16 * kK];
    }
    Acc sum = (t[0] + t[1]) + (t[2] + t[3]);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, 16);
    if (lane == 0 && r < s.rows) {
      Acc* y = static_cast<Acc*>(a.y) + (int64_t)j * a.ldy;
      Acc v = a.alpha_one ? sum : (Acc)a.alpha * sum;
      if (a.beta_nonzero) v = fma((Acc)a.beta, y[gr], v);
      y[gr] = v;
    }
  }
}

// Adds the parts of split block rows: blocks [0, nb_narrow) take rows with few parts (16
// threads per row), the remaining blocks one row with many parts each. One launch, a
// programmatic dependent of the run kernel: it waits until that grid has completed and
// its partial sums are visible (a no-op after an ordinary launch).
template <class Acc, int kMaxP, int kK>
__global__ void __launch_bounds__(256) combine_kernel(const __grid_constant__ BatchArgs<kMaxP> b, uint32_t nb_narrow) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (blockIdx.x < nb_narrow) combine_narrow<Acc, kMaxP, kK>(b, blockIdx.x);
  else combine_wide<Acc, kMaxP, kK>(b, blockIdx.x - nb_narrow);
}

// ---- lane-stream run kernel (FP64 values, layout in cb_layout.h) -------------------------
// Persistent grid, one CTA per SM; every warp is an independent worker that takes its CTA's
// units by ticket, like the record kernel. Per unit a warp
//   * gathers the unit's x values (16 per sub-block, through restore_cols when aggregated:
//     the x preload of Algorithms 3/4) into one of its two x buffers with cp.async, one unit
//     ahead, so the gather of the next unit overlaps the walk of this one;
//   * walks its lane runs: each step is one coalesced 8-byte value load per lane, one 16-bit
//     entry word (x slot and row) and one FP64 FMA into the lane's row accumulator; values
//     and words are loaded a group of 8 steps ahead into two register sets used in turn
//     (the next unit's first group while the last group of this unit is computed), so no
//     shared-memory staging of the matrix is needed;
//   * finishes rows that cross lane runs: the lane where a row ends adds the partial sums of
//     the lanes before it in lane order (a segmented scan when a row spans many lanes), and
//     writes y once per row (block rows cut into parts: 16 partial sums per part, added by
//     the combine kernel in part order). Results do not depend on scheduling.
#ifndef CB_LANE_WARPS
#define CB_LANE_WARPS 20       // worker warps per SM (measured on the FEM band: 16 -> 20 -> 24)
#endif
#ifndef CB_LANE_WARPS_LP
#define CB_LANE_WARPS_LP 32    // the same for the 2-byte value types (20 -> 24 -> 28 -> 32)
#endif
#ifndef CB_LANE_WARPS_F32
#define CB_LANE_WARPS_F32 28   // FP32 values (32 -> 28: FEM -1%, R-MAT -3.5%; registers 64 -> 73)
#endif
template <class V, int kK>
struct LaneGeom {
  using Acc = typename ValT<V>::Acc;
  static constexpr uint32_t kSlot = (uint32_t)sizeof(Acc) * kK;       // bytes of one x slot
  static constexpr uint32_t kXBuf = CB_LANE_SLOTS * kSlot;            // one x buffer
  static constexpr uint32_t kOffRow = 2 * kXBuf;                      // row sums, CB_R_MAX x kK
  static constexpr uint32_t kOffCv = kOffRow + CB_R_MAX * kSlot;      // carry values, 32 x kK
  static constexpr uint32_t kOffCr = kOffCv + CB_VLANES * kSlot;      // carry rows, 32
  static constexpr uint32_t kWarpBytes = align128(kOffCr + 4u * CB_VLANES);
  static constexpr uint32_t kFit = (kSmemMax - kHeaderBytes) / kWarpBytes;
  // the FP64 walk is bound by the FP64 FMA pipe (20 warps measured best); the reduced types'
  // walk by latency, where more warps per SM help (registers shrink to fit)
  static constexpr int kWant = sizeof(V) == 8 ? CB_LANE_WARPS : sizeof(V) == 4 ? CB_LANE_WARPS_F32 : CB_LANE_WARPS_LP;
  static_assert(kWant <= 32, "at most 1024 threads per CTA");
  static constexpr int kWarps = kFit < (uint32_t)kWant ? (int)kFit : kWant;
  static constexpr uint32_t kSmem = kHeaderBytes + kWarps * kWarpBytes;
  static_assert(kWarps >= 4, "lane kernel warp buffers too large");
};
constexpr int kLaneGroup = CB_LANE_GROUP;   // steps per prefetch group (two words of four entries)
#ifndef CB_LANE_BATCH
#define CB_LANE_BATCH 1        // groups per prefetch batch of the 4- and 2-byte value types
#endif
#ifndef CB_LANE_FASTROW
#define CB_LANE_FASTROW 1      // reduced types: one row test per group of 8 entries
#endif

// streaming loads of read-only data that bypass L1 (plain asm: the compiler may predicate
// and schedule them)
__device__ __forceinline__ double ldg_stream_f64(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint64_t ldg_stream_u64(const uint64_t* p) {
  uint64_t v;
  asm("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ldg_stream_v4(const void* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// 16 bytes into shared memory, the first src_bytes of them from global memory, the rest zero
__device__ __forceinline__ void cp_async_16(uint32_t dst_smem, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst_smem), "l"(src), "r"(src_bytes) : "memory");
}

// The values of one group of 8 steps of a lane, as loaded: FP64 eight doubles (one per
// step row), the reduced types their 16 or 32 contiguous bytes.
template <class V> struct LaneVals;
template <> struct LaneVals<double> {
  double v[kLaneGroup];
  __device__ __forceinline__ double at(int j) const { return v[j]; }
};
template <> struct LaneVals<float> {
  uint4 a, b;
  __device__ __forceinline__ float at(int j) const {
    const uint4& q = j < 4 ? a : b;
    const uint32_t w = (j & 3) == 0 ? q.x : (j & 3) == 1 ? q.y : (j & 3) == 2 ? q.z : q.w;
    return __uint_as_float(w);
  }
};
__device__ __forceinline__ uint32_t half_word(const uint4& a, int j) {
  const uint32_t w = (j >> 1) == 0 ? a.x : (j >> 1) == 1 ? a.y : (j >> 1) == 2 ? a.z : a.w;
  return (j & 1) ? w >> 16 : w & 0xffffu;
}
template <> struct LaneVals<__nv_bfloat16> {
  uint4 a;
  __device__ __forceinline__ float at(int j) const { return __uint_as_float(half_word(a, j) << 16); }
};
template <> struct LaneVals<__half> {
  uint4 a;
  __device__ __forceinline__ float at(int j) const {
    return __half2float(__ushort_as_half((unsigned short)half_word(a, j)));
  }
};

// Lane-stream run kernel (layout in cb_layout.h): a persistent CTA per SM; its warps take
// the CTA's units in turn. Per unit a warp gathers the unit's x values into shared memory
// (cp.async, one unit ahead), then every lane walks its run of entries with one FMA per
// entry, keeping the partial sum of its current row in a register; row sums go to
// shared memory, rows that cross lane runs are joined through the neighbouring lanes, and
// the unit's rows are written to y (or to the partial-sum slot of a block-row part).
template <class V, int kMaxP, int kK>
__global__ void __launch_bounds__(32 * LaneGeom<V, kK>::kWarps, 1)
    spmv_lanes_kernel(const __grid_constant__ BatchArgs<kMaxP> b) {
  using Acc = typename ValT<V>::Acc;
  using G = LaneGeom<V, kK>;
  constexpr bool kGrouped = sizeof(V) != 8;
  constexpr int kB = kGrouped ? CB_LANE_BATCH : 1;
  constexpr uint32_t kFull = 0xffffffffu;
  constexpr uint32_t kNone = 0xffffffffu;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  CtaHeader& hd = *reinterpret_cast<CtaHeader*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* W = smem_raw + kHeaderBytes + (uint32_t)warp * G::kWarpBytes;
  const uint32_t w_smem = smem_u32(W);
  Acc* srow = reinterpret_cast<Acc*>(W + G::kOffRow);
  Acc* cval = reinterpret_cast<Acc*>(W + G::kOffCv);
  int32_t* crow = reinterpret_cast<int32_t*>(W + G::kOffCr);
  // every CTA of this persistent grid is resident from the start, so the dependent combine
  // launch (if any) may be scheduled now: its CTAs take SMs as this grid's CTAs finish and
  // wait for the whole grid before reading the partial sums
  asm volatile("griddepcontrol.launch_dependents;");
  const int P = b.count;
  if ((int)threadIdx.x < P) {
    const RunArgs& a = b.p[threadIdx.x];
    const uint32_t w0 = a.worker_off[blockIdx.x];
    hd.first[threadIdx.x] = w0;
    hd.pref[threadIdx.x + 1] = a.worker_off[blockIdx.x + 1] - w0;
  }
  if (threadIdx.x == 0) hd.ticket = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    hd.pref[0] = 0;
    for (int q = 0; q < P; ++q) hd.pref[q + 1] += hd.pref[q];
  }
  __syncthreads();
  const uint32_t total = hd.pref[P];
  auto grab = [&]() -> uint32_t {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&hd.ticket, 1u);
    return __shfl_sync(kFull, t, 0);
  };
  auto problem_of = [&](uint32_t t) -> int {
    if (kMaxP == 1) return 0;
    int lo = 0, hi = P - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (hd.pref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  // the 32-byte descriptor of ticket t (every lane loads it: one broadcast request)
  auto fetch = [&](uint32_t t, int& q, CbLaneUnit& u) {
    q = problem_of(t);
    const uint4* d = reinterpret_cast<const uint4*>(b.p[q].lunits + hd.first[q] + (t - hd.pref[q]));
    const uint4 d0 = __ldg(d), d1 = __ldg(d + 1);
    u.vals = d0.x; u.words = d0.y; u.gcols = d0.z; u.brow_lo = d0.w;
    u.steps = (uint16_t)(d1.x & 0xffffu); u.nslots = (uint16_t)(d1.x >> 16);
    u.nrows = (uint16_t)(d1.y & 0xffffu); u.flags = (uint16_t)(d1.y >> 16);
    u.slot = d1.z; u.gbase = d1.w;
  };
  // cp.async of the unit's x values into buffer `buf`: slot k gets x[column of slot k] (kK
  // vectors side by side); slots outside [0, n) read zero. Plain sub-blocks: 16
  // consecutive x values per sub-block in 16-byte copies when x is 16-byte aligned.
  auto gather = [&](int q, const CbLaneUnit& u, uint32_t buf) {
    constexpr int kPer = CB_LANE_SLOTS / 32;
    const RunArgs& a = b.p[q];
    const Acc* x = static_cast<const Acc*>(a.x);
    const int32_t* gc = a.lgcols + u.gcols;
    const uint32_t dst = w_smem + buf * G::kXBuf;
    if (kGrouped && (u.flags & CB_LUNIT_PLAINX)) {   // (the FP64 layout keeps per-slot lists)
      const uint32_t nt = u.nslots / 16u;
      const int32_t c0 = (uint32_t)lane < nt ? __ldg(gc + lane) : 0;
      if (kK == 1 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
        constexpr uint32_t kPerChunk = 16u / sizeof(Acc);          // x values per 16-byte copy
        constexpr uint32_t kChunks = 16u / kPerChunk;              // copies per sub-block
        const uint32_t total_chunks = nt * kChunks;
        for (uint32_t k0 = 0; k0 < total_chunks; k0 += 32u) {
          const uint32_t k = k0 + (uint32_t)lane;
          const uint32_t t = k / kChunks, h = k % kChunks;
          const int32_t ct = __shfl_sync(kFull, c0, (int)(t & 31u));
          if (k < total_chunks) {
            const int64_t col = (int64_t)ct + h * kPerChunk;
            const int64_t left = a.n - col;
            const uint32_t nb = left <= 0 ? 0u : left >= (int64_t)kPerChunk ? 16u : (uint32_t)left * (uint32_t)sizeof(Acc);
            cp_async_16(dst + 16u * k, x + (nb ? col : 0), nb);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          const uint32_t k = (uint32_t)lane + 32u * i;
          const int32_t ct = __shfl_sync(kFull, c0, (int)((k / 16u) & 31u));
          if (k < u.nslots) {
            const int64_t col = (int64_t)ct + (k & 15u);
            const bool ok = col < a.n;
#pragma unroll
            for (int j = 0; j < kK; ++j)
              cp_async_elem<sizeof(Acc)>(dst + G::kSlot * k + (uint32_t)sizeof(Acc) * j,
                                         x + (ok ? col + j * a.ldx : 0), ok ? (uint32_t)sizeof(Acc) : 0u);
          }
        }
      }
      return;
    }
    int32_t c[kPer];
    if (u.flags & CB_LUNIT_G16) {   // uint16 offsets from gbase, 0xffff for none
      const uint16_t* g16 = reinterpret_cast<const uint16_t*>(gc);
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t k = (uint32_t)lane + 32u * i;
        const uint32_t o = k < u.nslots ? (uint32_t)__ldg(g16 + k) : 0xffffu;
        c[i] = o == 0xffffu ? -1 : (int32_t)(u.gbase + o);
      }
    } else {
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t k = (uint32_t)lane + 32u * i;
        c[i] = k < u.nslots ? __ldg(gc + k) : -1;
      }
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const uint32_t k = (uint32_t)lane + 32u * i;
      if (k < u.nslots) {
        const bool ok = c[i] >= 0 && (int64_t)c[i] < a.n;
#pragma unroll
        for (int j = 0; j < kK; ++j)
          cp_async_elem<sizeof(Acc)>(dst + G::kSlot * k + (uint32_t)sizeof(Acc) * j,
                                     x + (ok ? (int64_t)c[i] + j * a.ldx : 0), ok ? (uint32_t)sizeof(Acc) : 0u);
      }
    }
  };
  // this lane's value and word streams of a unit
  auto vbase = [&](int q, const CbLaneUnit& u) -> const V* {
    const V* v = static_cast<const V*>(b.p[q].lvals) + (size_t)u.vals * CB_VLANES;
    return kGrouped ? v + (uint32_t)lane * kLaneGroup : v + lane;
  };
  auto wbase = [&](int q, const CbLaneUnit& u) -> const uint64_t* {
    const uint64_t* w = b.p[q].lwords + (size_t)u.words * CB_VLANES;
    return kGrouped ? w + 2u * (uint32_t)lane : w + lane;
  };
  // values and entry words of steps 8g .. 8g + 7 (absent steps: no entry); plain loads the
  // compiler can predicate, with immediate offsets from the group's base
  auto load_group = [&](const V* vp, const uint64_t* wp, uint32_t S, uint32_t g, LaneVals<V>& v, uint64_t& w0,
                        uint64_t& w1) {
    const int rem = (int)S - (int)(kLaneGroup * g);
    if constexpr (!kGrouped) {
      const double* p = reinterpret_cast<const double*>(vp) + kLaneGroup * CB_VLANES * g;
#pragma unroll
      for (int j = 0; j < kLaneGroup; ++j)
        if (j < rem) v.v[j] = ldg_stream_f64(p + CB_VLANES * j);
      const uint64_t* pw = wp + 2u * CB_VLANES * g;
      w0 = rem > 0 ? ldg_stream_u64(pw) : ~0ull;
      w1 = rem > 4 ? ldg_stream_u64(pw + CB_VLANES) : ~0ull;
    } else {
      const V* p = vp + kLaneGroup * CB_VLANES * g;
      const uint64_t* pw = wp + 2u * CB_VLANES * g;
      if (rem >= kLaneGroup) {
        v.a = ldg_stream_v4(p);
        if constexpr (sizeof(V) == 4) v.b = ldg_stream_v4(p + 4);
        const uint4 ww = ldg_stream_v4(pw);
        w0 = ((uint64_t)ww.y << 32) | ww.x;
        w1 = ((uint64_t)ww.w << 32) | ww.z;
      } else if (rem > 0) {
        // the unit's last rem < 8 steps: each lane's rem values and ceil(rem / 4) words are
        // contiguous after the full groups (vp and wp point at this lane's full-group data)
        const int l = lane;
        const V* pt = p + l * (rem - kLaneGroup);
        uint32_t e[kLaneGroup];
#pragma unroll
        for (int j = 0; j < kLaneGroup; ++j) {
          e[j] = 0u;
          if (j < rem) {
            if constexpr (sizeof(V) == 4) e[j] = __ldg(reinterpret_cast<const uint32_t*>(pt) + j);
            else e[j] = (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(pt) + j);
          }
        }
        if constexpr (sizeof(V) == 4) {
          v.a = make_uint4(e[0], e[1], e[2], e[3]);
          v.b = make_uint4(e[4], e[5], e[6], e[7]);
        } else {
          v.a = make_uint4(e[0] | e[1] << 16, e[2] | e[3] << 16, e[4] | e[5] << 16, e[6] | e[7] << 16);
        }
        const uint64_t* pwt = pw + l * (rem > 4 ? 0 : -1);   // 2 words per lane, or 1
        if (rem > 4) {
          const uint4 ww = ldg_stream_v4(pwt);
          w0 = ((uint64_t)ww.y << 32) | ww.x;
          w1 = ((uint64_t)ww.w << 32) | ww.z;
        } else {
          w0 = __ldg(pwt);
          w1 = ~0ull;
        }
      } else {
        w0 = w1 = ~0ull;
      }
    }
  };

  uint32_t t = grab();
  if (t >= total) return;
  int q = 0, qn = 0;
  CbLaneUnit u, un{};
  fetch(t, q, u);
  gather(q, u, 0);
  cp_async_commit();
  // kB groups per prefetch batch: the reduced types' groups hold few bytes, so more of them
  // are kept in flight per warp
  struct Batch {
    LaneVals<V> v[kB];
    uint64_t w[2 * kB];
  };
  auto load_batch = [&](const V* vp, const uint64_t* wp, uint32_t S, uint32_t bi, Batch& bt) {
#pragma unroll
    for (int i = 0; i < kB; ++i) load_group(vp, wp, S, bi * kB + i, bt.v[i], bt.w[2 * i], bt.w[2 * i + 1]);
  };
  Batch ba, bb;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    if constexpr (!kGrouped) {
#pragma unroll
      for (int j = 0; j < kLaneGroup; ++j) ba.v[i].v[j] = bb.v[i].v[j] = 0.0;
    } else {
      ba.v[i].a = bb.v[i].a = make_uint4(0, 0, 0, 0);
      if constexpr (sizeof(V) == 4) ba.v[i].b = bb.v[i].b = make_uint4(0, 0, 0, 0);
    }
    bb.w[2 * i] = bb.w[2 * i + 1] = ~0ull;
  }
  load_batch(vbase(q, u), wbase(q, u), u.steps, 0, ba);
  uint32_t tn = grab();
  if (tn < total) fetch(tn, qn, un);
  uint32_t buf = 0;
  for (;;) {
    if (tn < total) gather(qn, un, buf ^ 1u);   // the next unit's x, during this unit's walk
    cp_async_commit();
    const uint32_t tnn = grab();
    int qnn = 0;
    CbLaneUnit unn{};
    if (tnn < total) fetch(tnn, qnn, unn);
    const RunArgs& a = b.p[q];
    const uint32_t R = u.nrows;
    for (uint32_t r = lane; r < R * kK; r += 32) srow[r] = (Acc)0;
    cp_async_wait_one();                       // this unit's x values have landed
    __syncwarp();
    const uint8_t* xs = W + buf * G::kXBuf;

    // walk
    Acc acc[kK], head[kK];
#pragma unroll
    for (int j = 0; j < kK; ++j) acc[j] = head[j] = (Acc)0;
    uint32_t cur = kNone, first_row = kNone;
    bool have_head = false;
    const uint32_t ngroups = (u.steps + kLaneGroup - 1u) / kLaneGroup;
    const V* vp = vbase(q, u);
    const uint64_t* wp = wbase(q, u);
    const V* vpn = tn < total ? vbase(qn, un) : vp;
    const uint64_t* wpn = tn < total ? wbase(qn, un) : wp;
    const uint32_t Sn = tn < total ? un.steps : 0u;
    // the entries of one group: x operands first (slot 511 of an absent entry lies inside the
    // buffer and is not used), then the FMA chain with the rare row switch
    auto compute = [&](const LaneVals<V>& v, uint64_t w0, uint64_t w1) {
#if CB_LANE_FASTROW
      if constexpr (kGrouped) {
        // the common case of the reduced types, whose walk is bound by instruction issue:
        // all 8 entries of the group continue the current row (row bits of every word
        // equal cur), so no row switch is tested per entry and two partial sums per vector
        // break the FMA dependency chain
        const uint64_t row_bits = 0xFE00FE00FE00FE00ull;
        const uint64_t pat = (uint64_t)cur * 0x0200020002000200ull;
        if (cur < 128u && (w0 & row_bits) == pat && (w1 & row_bits) == pat) {
          Acc s0[kK], s1[kK];
#pragma unroll
          for (int h = 0; h < kK; ++h) s0[h] = s1[h] = (Acc)0;
#pragma unroll
          for (int j = 0; j < kLaneGroup; ++j) {
            const uint32_t slot = (uint32_t)((j < 4 ? w0 : w1) >> (16 * (j & 3))) & 511u;
            const Acc vj = v.at(j);
            if constexpr (kK == 4) {   // the slot's four x values in one 16-byte load
              const float4 x4 = *reinterpret_cast<const float4*>(xs + G::kSlot * slot);
              const Acc xh[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                if (j & 1) s1[h] = fma(vj, xh[h], s1[h]); else s0[h] = fma(vj, xh[h], s0[h]);
              }
            } else {
#pragma unroll
              for (int h = 0; h < kK; ++h) {
                const Acc xj = *reinterpret_cast<const Acc*>(xs + G::kSlot * slot + sizeof(Acc) * h);
                if (j & 1) s1[h] = fma(vj, xj, s1[h]); else s0[h] = fma(vj, xj, s0[h]);
              }
            }
          }
#pragma unroll
          for (int h = 0; h < kK; ++h) acc[h] += s0[h] + s1[h];
          return;
        }
      }
#endif
      Acc xv[kLaneGroup][kK];
#pragma unroll
      for (int j = 0; j < kLaneGroup; ++j) {
        const uint32_t w = (uint32_t)((j < 4 ? w0 : w1) >> (16 * (j & 3))) & 0xffffu;
        const uint32_t slot = w & 511u;
        if constexpr (kK == 1) {
          xv[j][0] = *reinterpret_cast<const Acc*>(xs + (uint32_t)sizeof(Acc) * slot);
        } else {
#pragma unroll
          for (int h = 0; h < kK; ++h) xv[j][h] = *reinterpret_cast<const Acc*>(xs + G::kSlot * slot + sizeof(Acc) * h);
        }
      }
#pragma unroll
      for (int j = 0; j < kLaneGroup; ++j) {
        const uint32_t w = (uint32_t)((j < 4 ? w0 : w1) >> (16 * (j & 3))) & 0xffffu;
        const uint32_t r = w >> 9;
        if (r != cur && w != CB_LANE_NONE) {
          if (cur == kNone) {
            first_row = r;
          } else if (!have_head) {
#pragma unroll
            for (int h = 0; h < kK; ++h) head[h] = acc[h];
            have_head = true;
          } else {
#pragma unroll
            for (int h = 0; h < kK; ++h) srow[cur * kK + h] = acc[h];
          }
#pragma unroll
          for (int h = 0; h < kK; ++h) acc[h] = (Acc)0;
          cur = r;
        }
        if (w != CB_LANE_NONE) {
          const Acc vj = v.at(j);
#pragma unroll
          for (int h = 0; h < kK; ++h) acc[h] = fma(vj, xv[j][h], acc[h]);
        }
      }
    };
    auto compute_batch = [&](const Batch& bt) {
#pragma unroll
      for (int i = 0; i < kB; ++i) compute(bt.v[i], bt.w[2 * i], bt.w[2 * i + 1]);
    };
    // two register sets in turn: the batch after the current one (or the next unit's first
    // batch) is loaded while the current one is computed
    const uint32_t nbatch = (ngroups + kB - 1u) / kB;
    uint32_t g = 0;
    while (g < nbatch) {
      if (g + 1 < nbatch) load_batch(vp, wp, u.steps, g + 1, bb);
      else load_batch(vpn, wpn, Sn, 0, bb);
      compute_batch(ba);
      if (++g >= nbatch) {
        ba = bb;
        break;
      }
      if (g + 1 < nbatch) load_batch(vp, wp, u.steps, g + 1, ba);
      else load_batch(vpn, wpn, Sn, 0, ba);
      compute_batch(bb);
      ++g;
    }
    if (nbatch == 0) load_batch(vpn, wpn, Sn, 0, ba);   // (no entries) keep the prefetch in step

    // rows that cross lane runs: neighbours are the nearest lanes with entries
    const bool nonempty = cur != kNone;
    int prev = nonempty ? lane : -1, next = nonempty ? lane : 32;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(kFull, prev, d);
      if (lane >= d && o > prev) prev = o;
      const int p2 = __shfl_down_sync(kFull, next, d);
      if (lane + d < 32 && p2 < next) next = p2;
    }
    int prev_ne = __shfl_up_sync(kFull, prev, 1);
    int next_ne = __shfl_down_sync(kFull, next, 1);
    if (lane == 0) prev_ne = -1;
    if (lane == 31) next_ne = 32;
    const int32_t my_first = nonempty ? (int32_t)first_row : -1, my_last = nonempty ? (int32_t)cur : -1;
    const int32_t prev_last = __shfl_sync(kFull, my_last, prev_ne < 0 ? 0 : prev_ne);
    const int32_t next_first = __shfl_sync(kFull, my_first, next_ne > 31 ? 0 : next_ne);
    const bool hs = nonempty && prev_ne >= 0 && prev_last == my_first;     // first row began earlier
    const bool open = nonempty && next_ne <= 31 && next_first == my_last;  // last row continues
    int32_t own_row = -1, carry_row = -1;
    Acc own_val[kK], carry_val[kK];
#pragma unroll
    for (int h = 0; h < kK; ++h) own_val[h] = carry_val[h] = (Acc)0;
    if (nonempty) {
      if (have_head) {           // two or more rows in this run
        if (hs) {
          own_row = my_first;
#pragma unroll
          for (int h = 0; h < kK; ++h) own_val[h] = head[h];
        } else {
#pragma unroll
          for (int h = 0; h < kK; ++h) srow[my_first * kK + h] = head[h];
        }
        if (open) {
          carry_row = my_last;
#pragma unroll
          for (int h = 0; h < kK; ++h) carry_val[h] = acc[h];
        } else {
#pragma unroll
          for (int h = 0; h < kK; ++h) srow[my_last * kK + h] = acc[h];
        }
      } else if (open) {         // one row that continues (begun here or earlier)
        carry_row = my_last;
#pragma unroll
        for (int h = 0; h < kK; ++h) carry_val[h] = acc[h];
      } else if (hs) {           // one row begun earlier that ends here
        own_row = my_first;
#pragma unroll
        for (int h = 0; h < kK; ++h) own_val[h] = acc[h];
      } else {
#pragma unroll
        for (int h = 0; h < kK; ++h) srow[my_last * kK + h] = acc[h];
      }
    }
    if (!(u.flags & CB_LUNIT_SCAN)) {
      crow[lane] = nonempty ? carry_row : -2;
#pragma unroll
      for (int h = 0; h < kK; ++h) cval[lane * kK + h] = carry_val[h];
      __syncwarp();
      if (own_row >= 0) {
        Acc sum[kK];
#pragma unroll
        for (int h = 0; h < kK; ++h) sum[h] = own_val[h];
        for (int l = lane - 1; l >= 0; --l) {
          const int32_t cr = crow[l];
          if (cr == -2) continue;
          if (cr != own_row) break;
#pragma unroll
          for (int h = 0; h < kK; ++h) sum[h] += cval[l * kK + h];
        }
#pragma unroll
        for (int h = 0; h < kK; ++h) srow[own_row * kK + h] = sum[h];
      }
    } else {
      // segmented inclusive scan of the carries over lanes, keyed by the carried row; lanes
      // without entries take the key of the nearest lane with entries before them
      const int32_t key0 = nonempty ? carry_row : -2;
      const int32_t key = __shfl_sync(kFull, key0, prev < 0 ? lane : prev);
      Acc c2[kK];
#pragma unroll
      for (int h = 0; h < kK; ++h) c2[h] = carry_val[h];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t ko = __shfl_up_sync(kFull, key, d);
        const bool take = lane >= d && ko == key;
#pragma unroll
        for (int h = 0; h < kK; ++h) {
          const Acc vo = __shfl_up_sync(kFull, c2[h], d);
          if (take) c2[h] += vo;
        }
      }
      const int32_t kprev = __shfl_up_sync(kFull, key, 1);
#pragma unroll
      for (int h = 0; h < kK; ++h) {
        const Acc pv = __shfl_up_sync(kFull, c2[h], 1);
        if (own_row >= 0) srow[own_row * kK + h] = own_val[h] + (lane > 0 && kprev == own_row ? pv : (Acc)0);
      }
    }
    __syncwarp();

    // outputs (alpha and beta in the accumulation type)
    if (u.slot == 0xffffffffu) {
      Acc* y = static_cast<Acc*>(a.y);
      const Acc alpha = (Acc)a.alpha, beta = (Acc)a.beta;
      const int64_t row0 = (int64_t)u.brow_lo * CB_BLK;
      for (uint32_t r = lane; r < R; r += 32) {
#pragma unroll
        for (int h = 0; h < kK; ++h) {
          Acc* yh = y + (int64_t)h * a.ldy + row0 + r;
          Acc v = srow[r * kK + h];
          if (!a.alpha_one) v = alpha * v;
          if (a.beta_nonzero) v = fma(beta, *yh, v);
          *yh = v;
        }
      }
    } else {
      Acc* partial = static_cast<Acc*>(a.partial);
      if (lane < 16) {
#pragma unroll
        for (int h = 0; h < kK; ++h)
          partial[((size_t)u.slot * 16 + lane) * kK + h] = (uint32_t)lane < R ? srow[lane * kK + h] : (Acc)0;
      }
    }
    // the gather list of the unit after next into L2 (one bulk prefetch by the TMA unit
    // instead of scattered cold loads when its gather is issued)
    if (tnn < total && lane == 0 && unn.nslots) {
      const uint32_t ng = (kGrouped && (unn.flags & CB_LUNIT_PLAINX)) ? (unn.nslots / 16u + 3u) & ~3u
                          : (unn.flags & CB_LUNIT_G16) ? unn.nslots / 2u : unn.nslots;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b.p[qnn].lgcols + unn.gcols), "r"(4u * ng)
                   : "memory");
    }
    __syncwarp();
    if (tn >= total) break;
    t = tn; q = qn; u = un;
    tn = tnn; qn = qnn; un = unn;
    buf ^= 1u;
  }
  cp_async_wait_all();
}

// Raises the run kernel's dynamic shared-memory limit on the current device (once per
// device and instantiation).
// The flags are atomics: the server's engine thread and user threads launch concurrently.
// Two threads that both see a flag unset both set the (idempotent) attribute.
template <class V, int kMaxP, int kK>
cudaError_t configure_typed() {
  static std::atomic<bool> configured[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(spmv_kernel<V, kMaxP, kK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Geom<V, kK>::kSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev].store(true, std::memory_order_release);
  }
  return cudaSuccess;
}

template <class V, int kMaxP, int kK>
cudaError_t configure_lanes() {
  static std::atomic<bool> configured[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(spmv_lanes_kernel<V, kMaxP, kK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)LaneGeom<V, kK>::kSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev].store(true, std::memory_order_release);
  }
  return cudaSuccess;
}

// The kernels that add the parts of split block rows (after the run kernel, same stream).
template <class Acc, int kMaxP, int kK>
cudaError_t launch_combine(const BatchArgs<kMaxP>& b, cudaStream_t stream) {
  cudaError_t e = cudaSuccess;
  const uint32_t nsplit = b.split_base[b.count], nwide = b.wide_base[b.count];
  if (!nsplit && !nwide) return e;
  // one launch for both kinds of split rows, a programmatic dependent of the run kernel
  // (its launch overlaps the run kernel's tail)
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  const uint32_t nb_narrow = (16u * nsplit + 255u) / 256u;
  cfg.gridDim = dim3(nb_narrow + nwide);
  cfg.blockDim = dim3(256);
  cfg.stream = stream;
  cfg.attrs = pdl;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, combine_kernel<Acc, kMaxP, kK>, b, nb_narrow);
}

template <class V, int kMaxP, int kK>
cudaError_t launch_lanes(const BatchArgs<kMaxP>& b, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  using Acc = typename ValT<V>::Acc;
  using G = LaneGeom<V, kK>;
  cudaError_t e = configure_lanes<V, kMaxP, kK>();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) return e;
  spmv_lanes_kernel<V, kMaxP, kK><<<grid, 32 * G::kWarps, G::kSmem, stream>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) return e;
  e = launch_combine<Acc, kMaxP, kK>(b, stream);
  if (e != cudaSuccess) return e;
  if (ev) e = cudaEventRecord(ev[2], stream);
  return e;
}

template <class V, int kMaxP, int kK>
cudaError_t launch_typed(const BatchArgs<kMaxP>& b, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  using Acc = typename ValT<V>::Acc;
  const size_t smem = Geom<V, kK>::kSmem;
  cudaError_t e = configure_typed<V, kMaxP, kK>();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) return e;
  spmv_kernel<V, kMaxP, kK><<<grid, 32 * Geom<V, kK>::kWarps, smem, stream>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) return e;
  e = launch_combine<Acc, kMaxP, kK>(b, stream);
  if (e != cudaSuccess) return e;
  if (ev) e = cudaEventRecord(ev[2], stream);
  return e;
}

template <class V, int kMaxP>
cudaError_t launch_nvec(const BatchArgs<kMaxP>& b, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  if constexpr (kMaxP == 1) {     // several vectors per pass: single products only
    switch (b.p[0].nvec) {
      case 1: return launch_typed<V, 1, 1>(b, grid, stream, ev);
      case 2: return launch_typed<V, 1, 2>(b, grid, stream, ev);
      case 4: return launch_typed<V, 1, 4>(b, grid, stream, ev);
      default: return cudaErrorInvalidValue;
    }
  } else {   // batches: one vector, or passes of four
    return b.p[0].nvec == 1 ? launch_typed<V, kMaxP, 1>(b, grid, stream, ev)
           : b.p[0].nvec == 4 ? launch_typed<V, kMaxP, 4>(b, grid, stream, ev)
                              : cudaErrorInvalidValue;
  }
}

template <class V, int kMaxP>
cudaError_t launch_lanes_nvec(const BatchArgs<kMaxP>& b, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  // FP64: one vector per pass (the FP64 FMA pipe bounds the product; see cbspmv_run_multi);
  // the reduced types also in passes of four vectors, which read the streams once
  if constexpr (sizeof(V) != 8)
    if (b.p[0].nvec == 4) return launch_lanes<V, kMaxP, 4>(b, grid, stream, ev);
  return b.p[0].nvec == 1 ? launch_lanes<V, kMaxP, 1>(b, grid, stream, ev) : cudaErrorInvalidValue;
}

template <int kMaxP>
cudaError_t launch_dispatch(const BatchArgs<kMaxP>& b, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  if (b.p[0].lanes) {
    switch (b.p[0].value_dtype) {
      case CBSPMV_F64: return launch_lanes_nvec<double, kMaxP>(b, grid, stream, ev);
      case CBSPMV_F32: return launch_lanes_nvec<float, kMaxP>(b, grid, stream, ev);
      case CBSPMV_BF16: return launch_lanes_nvec<__nv_bfloat16, kMaxP>(b, grid, stream, ev);
      case CBSPMV_F16: return launch_lanes_nvec<__half, kMaxP>(b, grid, stream, ev);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (b.p[0].value_dtype) {
    case CBSPMV_F64: return launch_nvec<double, kMaxP>(b, grid, stream, ev);
    case CBSPMV_F32: return launch_nvec<float, kMaxP>(b, grid, stream, ev);
    case CBSPMV_BF16: return launch_nvec<__nv_bfloat16, kMaxP>(b, grid, stream, ev);
    case CBSPMV_F16: return launch_nvec<__half, kMaxP>(b, grid, stream, ev);
    default: return cudaErrorInvalidValue;
  }
}

// New values into the packed records: value k (CSR order, FP64) goes to value slot
// slot[k] of the stream, converted to the storage type like the analysis converts it.
__global__ void __launch_bounds__(256) repack_values_kernel(uint8_t* stream, const uint32_t* slot,
                                                            const double* val, int64_t nnz, int dtype) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
    const uint64_t bits = storage_bits(val[k], dtype);
    const size_t s = slot[k];
    switch (dtype) {
      case CBSPMV_F64: reinterpret_cast<uint64_t*>(stream)[s] = bits; break;
      case CBSPMV_F32: reinterpret_cast<uint32_t*>(stream)[s] = (uint32_t)bits; break;
      default: reinterpret_cast<uint16_t*>(stream)[s] = (uint16_t)bits; break;
    }
  }
}

}  // namespace

cudaError_t launch_repack(uint8_t* stream, const uint32_t* slot, const double* val, int64_t nnz, int dtype,
                          int grid, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  const int64_t blocks = (nnz + 255) / 256;
  repack_values_kernel<<<(int)(blocks < 8 * (int64_t)grid ? blocks : 8 * (int64_t)grid), 256, 0, s>>>(
      stream, slot, val, nnz, dtype);
  return cudaGetLastError();
}

size_t spmv_smem_bytes() {
  const uint32_t v[] = {Geom<double>::kSmem, Geom<float>::kSmem, Geom<__half>::kSmem, Geom<double, 4>::kSmem,
                        Geom<float, 4>::kSmem, Geom<__half, 4>::kSmem, LaneGeom<double, 1>::kSmem,
                        LaneGeom<float, 1>::kSmem, LaneGeom<__nv_bfloat16, 1>::kSmem, LaneGeom<float, 4>::kSmem};
  uint32_t m = 0;
  for (uint32_t x : v) m = x > m ? x : m;
  return m;
}
int spmv_warps(int value_dtype) {
  switch (value_dtype) {
    case CBSPMV_F64: return Geom<double>::kWarps;
    case CBSPMV_F32: return Geom<float>::kWarps;
    default: return Geom<__half>::kWarps;
  }
}

template <class V>
cudaError_t configure_value_type() {
  cudaError_t e = configure_typed<V, 1, 1>();
  if (e == cudaSuccess) e = configure_typed<V, kMaxBatch, 1>();
  if (e == cudaSuccess) e = configure_typed<V, kMaxBatch, 4>();
  if (e == cudaSuccess) e = configure_typed<V, 1, 2>();
  if (e == cudaSuccess) e = configure_typed<V, 1, 4>();
  return e;
}

cudaError_t configure_kernels() {
  cudaError_t e = configure_lanes<double, 1, 1>();
  if (e == cudaSuccess) e = configure_lanes<double, kMaxBatch, 1>();
  if (e == cudaSuccess) e = configure_lanes<float, 1, 1>();
  if (e == cudaSuccess) e = configure_lanes<float, kMaxBatch, 1>();
  if (e == cudaSuccess) e = configure_lanes<__nv_bfloat16, 1, 1>();
  if (e == cudaSuccess) e = configure_lanes<__nv_bfloat16, kMaxBatch, 1>();
  if (e == cudaSuccess) e = configure_lanes<__half, 1, 1>();
  if (e == cudaSuccess) e = configure_lanes<__half, kMaxBatch, 1>();
  if (e == cudaSuccess) e = configure_value_type<double>();
  if (e == cudaSuccess) e = configure_value_type<float>();
  if (e == cudaSuccess) e = configure_value_type<__nv_bfloat16>();
  if (e == cudaSuccess) e = configure_value_type<__half>();
  return e;
}

cudaError_t launch_spmv(const RunArgs& a, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  BatchArgs<1> b;
  b.count = 1;
  b.split_base[0] = 0;
  b.split_base[1] = a.n_split_rows - a.n_split_wide;
  b.wide_base[0] = 0;
  b.wide_base[1] = a.n_split_wide;
  b.p[0] = a;
  return launch_dispatch<1>(b, grid, stream, ev);
}

cudaError_t launch_spmv_batch(const RunArgs* a, int count, int grid, cudaStream_t stream) {
  for (int i = 0; i < count; ++i)
    if (a[i].value_dtype != a[0].value_dtype || a[i].nvec != a[0].nvec || (a[i].nvec != 1 && a[i].nvec != 4))
      return cudaErrorInvalidValue;
  // a single problem takes the single-product instantiation: the same arithmetic (so the
  // same result), without the 64-problem argument block or the problem lookup
  if (count == 1) return launch_spmv(a[0], grid, stream);
  // one layout per launch: problems of the other layout go to launches of their own
  for (int i = 1; i < count; ++i)
    if (a[i].lanes != a[0].lanes) {
      std::vector<RunArgs> l, r;
      for (int k = 0; k < count; ++k) (a[k].lanes ? l : r).push_back(a[k]);
      cudaError_t e = launch_spmv_batch(l.data(), (int)l.size(), grid, stream);
      return e == cudaSuccess ? launch_spmv_batch(r.data(), (int)r.size(), grid, stream) : e;
    }
  for (int base = 0; base < count; base += kMaxBatch) {
    const int c = count - base < kMaxBatch ? count - base : kMaxBatch;
    static thread_local BatchArgs<kMaxBatch> b;
    b.count = c;
    b.split_base[0] = 0;
    b.wide_base[0] = 0;
    for (int i = 0; i < c; ++i) {
      b.p[i] = a[base + i];
      b.split_base[i + 1] = b.split_base[i] + (a[base + i].n_split_rows - a[base + i].n_split_wide);
      b.wide_base[i + 1] = b.wide_base[i] + a[base + i].n_split_wide;
    }
    const cudaError_t e = launch_dispatch<kMaxBatch>(b, grid, stream, nullptr);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cb
