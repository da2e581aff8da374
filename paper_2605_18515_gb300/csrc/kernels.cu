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
// the FP64 pipe is the scarce unit (a warp-wide DFMA occupies it for ~19 cycles per SM
// and lanes that are masked off cost the same), so this kernel keeps the data structure
// and the per-tile decoding of the paper but reorganises the work:
//
//   * Persistent grid, one CTA per SM: kLoaders loader warps and CB_CONSUMERS consumer
//     warps. Loaders stage each unit of work (a run of consecutive tiles) into a ring of
//     CB_STAGES shared-memory stages with two bulk TMA copies (cp.async.bulk): the unit's
//     packed records and its blob (tile records, restore_cols slice, lane schedule). They
//     then gather the unit's x values into the stage with cp.async (the x preload of
//     Algorithms 3/4, through restore_cols for aggregated tiles); mbarriers hand stages to
//     the consumers and back. A consumer computes each tile's base addresses from its
//     record (CSR row pointer, COO coordinate bytes of Algorithm 3, the fixed rows of
//     Algorithm 4).
//   * The analyser's lane schedule cuts the unit's entries, in row-major order, into
//     chunks of at most CB_CHUNK entries of one (tile, row) piece and deals them to the
//     32 lanes in equal runs. Every lane then runs the same number of steps; a step reads
//     one 16-bit chunk descriptor, decodes up to three coordinate bytes and issues up to
//     three DFMAs into the lane's row accumulator. No FP64 work is spent on reductions:
//     a row sum is stored when its last chunk is done.
//   * Rows that cross run boundaries are completed by the run holding the row's end
//     (adding the earlier runs' carries in a fixed order); units that cover whole block
//     rows write y directly (no atomics, y read once when beta != 0). Block rows cut into
//     several units store 16 partial sums per part; a second small kernel adds the parts
//     in part order and writes y, so results do not depend on scheduling.
//   * Every wait is bounded (clock64 budget); on expiry the kernel records an error code,
//     drains its own copies in flight and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cb_layout.h"
#include "cb_kernels.h"

namespace cb {
namespace {

constexpr int kStages = CB_STAGES;
constexpr int kConsumers = CB_CONSUMERS;
constexpr int kLoaders = 4;                       // warps 0..3: bulk copies and x gather
constexpr int kProducers = kLoaders;
constexpr int kThreads = 32 * (kProducers + kConsumers);
constexpr long long kWaitBudget = 4000000000LL;   // clock64 cycles (~2 s) per wait

// Stage layout (byte offsets): the unit descriptor, the unit's packed records, its blob
// (tile records, restore_cols slice, lane schedule) and the gathered x values (16 per tile).
constexpr uint32_t kOffUnit = 0;
constexpr uint32_t kOffStream = 64;
constexpr uint32_t kOffBlob = kOffStream + CB_B_MAX;
constexpr uint32_t kBlobMax = 16 * CB_T_MAX + 4 * CB_RC_MAX + CB_SCHED_MAX;
constexpr uint32_t kOffXs = kOffBlob + kBlobMax;
constexpr uint32_t kStageBytes = (kOffXs + CB_T_MAX * 16 * 8 + 127) & ~127u;
static_assert(sizeof(CbUnit) == 64, "unit descriptor slot");
static_assert(kOffStream % 16 == 0 && kOffBlob % 16 == 0 && kOffXs % 16 == 0 && kBlobMax % 16 == 0,
              "bulk copy destinations must be 16-byte aligned");

// Stored value types: V is the storage type, Acc the type of x, y and the accumulators.
template <class V> struct ValT;
template <> struct ValT<double> {
  using Acc = double;
  __device__ static __forceinline__ double load(const uint8_t* p) { return *reinterpret_cast<const double*>(p); }
};
template <> struct ValT<float> {
  using Acc = float;
  __device__ static __forceinline__ float load(const uint8_t* p) { return *reinterpret_cast<const float*>(p); }
};
template <> struct ValT<__nv_bfloat16> {
  using Acc = float;
  __device__ static __forceinline__ float load(const uint8_t* p) {   // exact: bf16 is the top half of fp32
    return __uint_as_float((uint32_t)*reinterpret_cast<const uint16_t*>(p) << 16);
  }
};
template <> struct ValT<__half> {
  using Acc = float;
  __device__ static __forceinline__ float load(const uint8_t* p) {   // exact widening
    return __half2float(*reinterpret_cast<const __half*>(p));
  }
};

template <class Acc>
struct Scratch {
  uint4 tinfo[CB_T_MAX];        // per tile: value base, coordinate base, x-row base (smem offsets)
  Acc srow[CB_R_MAX];           // row sums
  Acc cval[CB_VLANES];          // per-run carry value
  int32_t crow[CB_VLANES];      // per-run carry row (-1 none, -2 no chunks)
};

template <class Acc>
struct Shared {
  __align__(128) uint8_t stage[kStages][kStageBytes];
  uint64_t bar_tma[kStages];    // bulk copies of the unit landed
  uint64_t bar_full[kStages];   // x gathered (the 32 lanes of a loader)
  // Exact hand-off words: the ticket whose copies were issued into the stage and the last
  // ticket released from it. Loaders issue their tickets out of order, so a stage's
  // barriers can be more than one phase behind a waiter; a waiter therefore first waits
  // for the exact ticket here, after which the parity waits are unambiguous.
  uint32_t issued[kStages];
  uint32_t released[kStages];
  Scratch<Acc> scratch[kConsumers];
  uint8_t ident[256];           // byte k = (k & 15) << 4: coordinate bytes of a Dense record
  uint32_t ticket;
  uint32_t abort_flag;
};

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
// Bounded wait until *p == v: false when the budget ran out.
__device__ __forceinline__ bool wait_value(const uint32_t* p, uint32_t v) {
  const volatile uint32_t* vp = p;
  if (*vp == v) return true;
  long long t0 = clock64();
  while (*vp != v) {
    __nanosleep(32);
    if (clock64() - t0 > kWaitBudget) return false;
  }
  return true;
}
// Bounded wait: false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitBudget) return false;
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
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t align16u(uint32_t v) { return (v + 15u) & ~15u; }

__device__ void set_error(const RunArgs& a, uint32_t code) { atomicOr(a.err, code); }

// ---- loader warps ------------------------------------------------------------------------
// Loader l (l = 0 .. kLoaders-1) owns tickets l, l + kLoaders, ...: for each it stores the
// unit descriptor in the stage and issues two bulk copies (packed records, unit blob) one
// ticket ahead, then gathers the current ticket's x values with cp.async (all 16 per tile;
// columns through restore_cols when aggregated) and signals the consumer through the
// stage's full barrier. Bulk copies issued by one thread complete one after another, so
// the copies are spread over several loader warps.
__device__ __forceinline__ uint32_t load_desc_word(const CbUnit* units, uint32_t k, uint32_t nu, int lane) {
  return (k < nu && lane < 16) ? __ldg(reinterpret_cast<const uint32_t*>(units + k) + lane) : 0u;
}

template <class Acc>
__device__ bool loader_issue(const RunArgs& a, Shared<Acc>& sh, uint32_t k, uint32_t dw, int lane) {
  const uint32_t s = k % kStages;
  // the stage's previous ticket (k - kStages) must have been released by its consumer
  if (k >= (uint32_t)kStages && !wait_value(&sh.released[s], k - kStages)) return false;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  uint8_t* S = sh.stage[s];
  if (lane < 16) reinterpret_cast<uint32_t*>(S + kOffUnit)[lane] = dw;
  __syncwarp();
  if (lane == 0) {
    *(volatile uint32_t*)&sh.issued[s] = k;
    const CbUnit& u = *reinterpret_cast<const CbUnit*>(S + kOffUnit);
    mbar_arrive_expect_tx(&sh.bar_tma[s], u.nbytes + u.blob_bytes);
    if (u.nbytes) bulk_g2s(S + kOffStream, a.stream + (size_t)u.byte_lo16 * 16, u.nbytes, &sh.bar_tma[s]);
    if (u.blob_bytes) bulk_g2s(S + kOffBlob, a.blob + (size_t)u.blob16 * 16, u.blob_bytes, &sh.bar_tma[s]);
  }
  __syncwarp();
  return true;
}

template <class Acc>
__device__ void loader(const RunArgs& a, Shared<Acc>& sh, const CbUnit* units, uint32_t nu, uint32_t l, int lane) {
  constexpr int kPerLane = CB_T_MAX * 16 / 32;
  constexpr uint32_t kXs = sizeof(Acc);
  const Acc* x = static_cast<const Acc*>(a.x);
  bool ok = true;
  uint32_t next = l;                                      // next own ticket to issue
  uint32_t dw = load_desc_word(units, next, nu, lane);    // its descriptor (16 lanes, one word each)
  if (next < nu) {
    ok = loader_issue(a, sh, next, dw, lane);
    next += kLoaders;
    dw = load_desc_word(units, next, nu, lane);
  }
  for (uint32_t j = l; j < nu && ok; j += kLoaders) {
    const uint32_t s = j % kStages, q = j / kStages;
    if (!mbar_wait(&sh.bar_tma[s], q & 1) || *(volatile uint32_t*)&sh.abort_flag) { ok = false; break; }
    const uint8_t* S = sh.stage[s];
    const CbUnit& u = *reinterpret_cast<const CbUnit*>(S + kOffUnit);
    const CbTile* tiles = reinterpret_cast<const CbTile*>(S + kOffBlob);
    const int32_t* rcols = reinterpret_cast<const int32_t*>(S + kOffBlob + 16u * u.ntiles);
    const uint32_t xs_smem = smem_u32(S + kOffXs);
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
        cp_async_elem<kXs>(xs_smem + kXs * idx, x + (valid ? col[k] : 0), valid ? kXs : 0u);
      }
    }
    cp_async_arrive_noinc(&sh.bar_full[s]);
    if (next < nu) {            // then keep one own ticket in flight ahead of the consumers
      ok = loader_issue(a, sh, next, dw, lane);
      next += kLoaders;
      dw = load_desc_word(units, next, nu, lane);
    }
  }
  if (!ok) {
    if (lane == 0) set_error(a, 1u);
    *(volatile uint32_t*)&sh.abort_flag = 1;
    // drain: copies of this loader's tickets issued but not waited for
    for (uint32_t k = l; k < next && k < nu; k += kLoaders)
      if (k + kStages >= next) mbar_wait(&sh.bar_tma[k % kStages], (k / kStages) & 1);
  }
  cp_async_wait_all();
}

// ---- consumer -----------------------------------------------------------------------------
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
#define CB_LDV(off) (ValT<V>::load(sm + (off)))
#define CB_LDX(off) (*reinterpret_cast<const Acc*>(sm + (off)))

// sm: base of the CTA's shared memory; so: offset of the unit's stage in it.
template <class V>
__device__ void consume_unit(const RunArgs& a, uint8_t* sm, uint32_t so, uint32_t ident_off,
                             Scratch<typename ValT<V>::Acc>& sc, int lane) {
  using Acc = typename ValT<V>::Acc;
  constexpr uint32_t kVs = sizeof(V), kXs = sizeof(Acc);
  // byte offset of x[col] in the tile's x row for a coordinate byte b (col = b >> 4)
  constexpr uint32_t kXShift = kXs == 8 ? 1 : 2, kXMask = 15u * kXs;
  uint8_t* S = sm + so;
  const CbUnit& u = *reinterpret_cast<const CbUnit*>(S + kOffUnit);
  const uint32_t T = u.ntiles;
  const uint32_t byte_lo = u.byte_lo16 * 16u;
  const int64_t row0 = (int64_t)u.brow_lo * CB_BLK;
  const int64_t rows_left = a.m - row0;
  const int64_t rows_unit = (int64_t)CB_BLK * u.nbr;
  const uint32_t R = (uint32_t)(rows_unit < rows_left ? rows_unit : rows_left);
  const CbTile* tiles = reinterpret_cast<const CbTile*>(S + kOffBlob);

  // 1. per-tile bases (lane = tile) and zeroed row sums
  if ((uint32_t)lane < T) {
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
    sc.tinfo[lane] = make_uint4(vb, cb, so + kOffXs + 16u * kXs * lane, 0u);
  }
  for (uint32_t r = lane; r < R; r += 32) sc.srow[r] = Acc(0);
  __syncwarp();

  // 2. one run per lane: a sequence of chunks of up to three entries; even chunks go to
  //    accumulator a0, odd chunks to a1 (two independent FP64 chains)
  const uint8_t* sched = S + kOffBlob + 16u * T + 4u * u.rc_n;
  const uint16_t* hdr = reinterpret_cast<const uint16_t*>(sched);
  const uint8_t* nxt = sched + 2 * CB_VLANES;
  const uint16_t* desc = reinterpret_cast<const uint16_t*>(sched + CB_SCHED_HDR(R));
  const uint32_t h = hdr[lane];
  const uint32_t nch = h >> 9;
  const uint32_t nmax = __reduce_max_sync(0xffffffffu, nch);
  const uint32_t steps = (nmax + 1) / 2;
  uint32_t row = h & 0xffu;
  const bool hs = (h >> 8) & 1u;
  bool first = true, open = false;
  int32_t own_row = -1;
  Acc own_val = Acc(0);
  Acc a0 = Acc(0), a1 = Acc(0);
  // Software pipeline: the operands of step i + 1 are loaded before the DFMAs of step i.
  // Loads are unconditional (a chunk shorter than three entries reads at most two entries
  // past its piece and column nibbles stay inside the tile's x row, so every address stays
  // in shared memory); the DFMA slots beyond the chunk's length are predicated off.
  uint32_t dA = 0, dB = 0;
  Acc vA0 = 0, vA1 = 0, vA2 = 0, xA0 = 0, xA1 = 0, xA2 = 0;
  Acc vB0 = 0, vB1 = 0, vB2 = 0, xB0 = 0, xB1 = 0, xB2 = 0;
#define CB_LOAD_CHUNK(d, v0, v1, v2, x0, x1, x2)                                   \
  {                                                                                \
    const uint4 ti_ = sc.tinfo[(d) & 31u];                                         \
    const uint32_t o_ = ((d) >> 5) & 255u;                                         \
    const uint32_t va_ = ti_.x + kVs * o_, ca_ = ti_.y + o_, xr_ = ti_.z;          \
    const uint32_t b0_ = sm[ca_], b1_ = sm[ca_ + 1], b2_ = sm[ca_ + 2];            \
    v0 = CB_LDV(va_);                                                              \
    v1 = CB_LDV(va_ + kVs);                                                        \
    v2 = CB_LDV(va_ + 2u * kVs);                                                   \
    x0 = CB_LDX(xr_ + ((b0_ >> kXShift) & kXMask));                                \
    x1 = CB_LDX(xr_ + ((b1_ >> kXShift) & kXMask));                                \
    x2 = CB_LDX(xr_ + ((b2_ >> kXShift) & kXMask));                                \
  }
  if (steps) {
    dA = desc[lane];
    dB = desc[CB_VLANES + lane];
    CB_LOAD_CHUNK(dA, vA0, vA1, vA2, xA0, xA1, xA2);
    CB_LOAD_CHUNK(dB, vB0, vB1, vB2, xB0, xB1, xB2);
  }
  for (uint32_t i = 0; i < steps; ++i) {
    const uint32_t nb = (i + 1 < steps ? 2u * (i + 1) : 2u * i) * CB_VLANES;
    const uint32_t dA_n = desc[nb + lane], dB_n = desc[nb + CB_VLANES + lane];
    Acc nvA0, nvA1, nvA2, nxA0, nxA1, nxA2, nvB0, nvB1, nvB2, nxB0, nxB1, nxB2;
    CB_LOAD_CHUNK(dA_n, nvA0, nvA1, nvA2, nxA0, nxA1, nxA2);
    CB_LOAD_CHUNK(dB_n, nvB0, nvB1, nvB2, nxB0, nxB1, nxB2);
    const uint32_t lA = (dA >> 13) & 3u, lB = (dB >> 13) & 3u;
    const bool eA = (dA & 0x8000u) != 0, eB = (dB & 0x8000u) != 0;
    // chunk B starts a new row when chunk A ends one: its chain then starts from zero
    const Acc a1_old = a1;
    Acc b = eA ? Acc(0) : a1;
    a0 = pfma(lA > 0, vA0, xA0, a0);
    b = pfma(lB > 0, vB0, xB0, b);
    a0 = pfma(lA > 1, vA1, xA1, a0);
    b = pfma(lB > 1, vB1, xB1, b);
    a0 = pfma(lA > 2, vA2, xA2, a0);
    b = pfma(lB > 2, vB2, xB2, b);
    a1 = b;
    if (lA | lB) open = true;
    if (eA) {                              // chunk A ends its row: a0 + (a1 before chunk B)
      const Acc sum = a0 + a1_old;
      if (first && hs) { own_row = (int32_t)row; own_val = sum; }
      else sc.srow[row] = sum;
      first = false;
      a0 = Acc(0);
      open = lB != 0;
      row = nxt[row];
    }
    if (eB) {                              // chunk B ends its row
      const Acc sum = a0 + a1;
      if (first && hs) { own_row = (int32_t)row; own_val = sum; }
      else sc.srow[row] = sum;
      first = false;
      a0 = Acc(0);
      a1 = Acc(0);
      open = false;
      row = nxt[row];
    }
    dA = dA_n;
    dB = dB_n;
    vA0 = nvA0; vA1 = nvA1; vA2 = nvA2; xA0 = nxA0; xA1 = nxA1; xA2 = nxA2;
    vB0 = nvB0; vB1 = nvB1; vB2 = nvB2; xB0 = nxB0; xB1 = nxB1; xB2 = nxB2;
  }
#undef CB_LOAD_CHUNK
  sc.crow[lane] = nch == 0 ? -2 : (open ? (int32_t)row : -1);
  sc.cval[lane] = open ? a0 + a1 : Acc(0);
  __syncwarp();
  if (own_row >= 0) {
    Acc sum = own_val;
    for (int j = (int)lane - 1; j >= 0; --j) {
      const int32_t cr = sc.crow[j];
      if (cr == -2) continue;
      if (cr != own_row) break;
      sum += sc.cval[j];
    }
    sc.srow[own_row] = sum;
  }
  __syncwarp();

  // 3. outputs (alpha and beta in the accumulation type)
  const Acc alpha = (Acc)a.alpha, beta = (Acc)a.beta;
  Acc* y = static_cast<Acc*>(a.y);
  if (u.split < 0) {
    for (uint32_t r = lane; r < R; r += 32) {
      const int64_t gr = row0 + r;
      Acc v = sc.srow[r];
      if (!a.alpha_one) v = alpha * v;
      if (a.beta_nonzero) v = fma(beta, y[gr], v);
      y[gr] = v;
    }
  } else {
    // part of a block row cut into several units: 16 partial sums, added by combine_kernel
    Acc* partial = static_cast<Acc*>(a.partial);
    if (lane < 16) partial[(size_t)u.slot * 16 + lane] = (uint32_t)lane < R ? sc.srow[lane] : Acc(0);
  }
}
#undef CB_LDV
#undef CB_LDX

template <class V>
__global__ void __launch_bounds__(kThreads, 1) spmv_kernel(const RunArgs a) {
  using Acc = typename ValT<V>::Acc;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Shared<Acc>& sh = *reinterpret_cast<Shared<Acc>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t w0 = a.worker_off[blockIdx.x], w1 = a.worker_off[blockIdx.x + 1];
  const CbUnit* units = a.units + w0;   // this CTA's units, stored contiguously
  const uint32_t nu = w1 - w0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh.bar_tma[s], 1);
      mbar_init(&sh.bar_full[s], 32);
      sh.issued[s] = 0xffffffffu;
      sh.released[s] = 0xffffffffu;
    }
    sh.ticket = 0;
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (uint32_t i = threadIdx.x; i < 256u; i += blockDim.x) sh.ident[i] = (uint8_t)((i & 15u) << 4);
  __syncthreads();
  if (warp < kLoaders) {
    loader(a, sh, units, nu, (uint32_t)warp, lane);
    return;
  }
  Scratch<Acc>& sc = sh.scratch[warp - kProducers];
  const uint32_t ident_off = (uint32_t)(sh.ident - smem_raw);
  for (;;) {
    uint32_t j = 0;
    if (lane == 0) j = atomicAdd(&sh.ticket, 1u);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= nu) break;
    const uint32_t s = j % kStages, q = j / kStages;
    bool ok = wait_value(&sh.issued[s], j);    // the stage now holds ticket j's copies
    ok = ok && mbar_wait(&sh.bar_full[s], q & 1);
    ok = ok && mbar_wait(&sh.bar_tma[s], q & 1);
    if (!__all_sync(0xffffffffu, ok) || *(volatile uint32_t*)&sh.abort_flag) {
      if (lane == 0) set_error(a, 2u);
      break;
    }
    consume_unit<V>(a, smem_raw, (uint32_t)(sh.stage[s] - smem_raw), ident_off, sc, lane);
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      *(volatile uint32_t*)&sh.released[s] = j;
    }
  }
}

// Adds the parts of every block row cut into several units, in part order, and writes y.
template <class Acc>
__global__ void __launch_bounds__(256) combine_kernel(const RunArgs a) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t sr = g >> 4, r = g & 15u;
  if (sr >= a.n_split_rows) return;
  const CbSplitRow s = a.split_rows[sr];
  if (r >= s.rows) return;
  const Acc* p = static_cast<const Acc*>(a.partial) + (size_t)s.slot0 * 16 + r;
  Acc sum = Acc(0);
  for (uint32_t k = 0; k < s.nparts; ++k) sum += p[(size_t)k * 16];
  const int64_t gr = (int64_t)s.brow * CB_BLK + r;
  Acc* y = static_cast<Acc*>(a.y);
  Acc v = a.alpha_one ? sum : (Acc)a.alpha * sum;
  if (a.beta_nonzero) v = fma((Acc)a.beta, y[gr], v);
  y[gr] = v;
}

template <class V>
cudaError_t launch_typed(const RunArgs& a, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  using Acc = typename ValT<V>::Acc;
  static bool configured[64] = {false};
  const size_t smem = sizeof(Shared<Acc>);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(spmv_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  if (ev && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) return e;
  spmv_kernel<V><<<grid, kThreads, smem, stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) return e;
  if (a.n_split_rows) {
    const uint32_t threads = 16u * a.n_split_rows;
    combine_kernel<Acc><<<(threads + 255) / 256, 256, 0, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ev) e = cudaEventRecord(ev[2], stream);
  return e;
}

}  // namespace

size_t spmv_smem_bytes() { return sizeof(Shared<double>) > sizeof(Shared<float>) ? sizeof(Shared<double>) : sizeof(Shared<float>); }
int spmv_threads() { return kThreads; }

cudaError_t launch_spmv(const RunArgs& a, int grid, cudaStream_t stream, cudaEvent_t* ev) {
  switch (a.value_dtype) {
    case CBSPMV_F64: return launch_typed<double>(a, grid, stream, ev);
    case CBSPMV_F32: return launch_typed<float>(a, grid, stream, ev);
    case CBSPMV_BF16: return launch_typed<__nv_bfloat16>(a, grid, stream, ev);
    case CBSPMV_F16: return launch_typed<__half>(a, grid, stream, ev);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cb
