// Run kernel of the blocked SpMV, y = alpha * A * x + beta * y, FP64, for sm_103a.
//
// The paper's kernel (Sec. 3.5, Algorithms 3 and 4) maps one sub-block to one warp,
// preloads x into shared memory (plain tiles) or reads it through restore_cols
// (aggregated tiles), reduces with warp shuffles and adds into y with atomics. On GB300
// the FP64 pipe is the scarce unit (a warp-wide DFMA occupies it for ~19 cycles per SM
// and lanes that are masked off cost the same), so this kernel keeps the data structure
// and the per-tile decoding of the paper but reorganises the work:
//
//   * Persistent grid, one CTA per SM: warp 0 is the producer, warps 1..CB_CONSUMERS are
//     consumers. One producer lane stages each unit of work (a run of consecutive tiles)
//     into a ring of CB_STAGES shared-memory stages with bulk TMA copies (cp.async.bulk)
//     of the unit's packed records, tile records and restore_cols slice; mbarriers hand
//     stages between the producer and the consumers.
//   * A consumer first gathers the unit's x values into the stage with cp.async (the x
//     preload of Algorithms 3/4, through restore_cols for aggregated tiles) and computes
//     each tile's base addresses from its record (CSR row pointer, COO coordinate bytes
//     of Algorithm 3, the fixed rows of Algorithm 4).
//   * The analyser's lane schedule cuts the unit's entries, in row-major order, into
//     chunks of at most CB_CHUNK entries of one (tile, row) piece and deals them to the
//     32 lanes in equal runs. Every lane then runs the same number of steps; a step reads
//     one 16-bit chunk descriptor, decodes up to three coordinate bytes and issues up to
//     three DFMAs into the lane's row accumulator. No FP64 work is spent on reductions:
//     a row sum is stored when its last chunk is done.
//   * Rows that cross lane boundaries are completed by the lane holding the row's end
//     (adding its neighbours' carries in a fixed order); units that cover whole block rows
//     write y directly (no atomics, y read once when beta != 0). Block rows cut into
//     several units combine their parts through a partial-sum buffer: the last part to
//     arrive (atomic counter) adds the parts in part order and writes y, so results do
//     not depend on scheduling.
//   * Every wait is bounded (clock64 budget); on expiry the kernel records an error code,
//     drains its own copies in flight and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cb_layout.h"
#include "cb_kernels.h"

namespace cb {
namespace {

constexpr int kStages = CB_STAGES;
constexpr int kConsumers = CB_CONSUMERS;
constexpr int kThreads = 32 * (1 + kConsumers);
constexpr long long kWaitBudget = 4000000000LL;   // clock64 cycles (~2 s) per wait

// Stage layout (byte offsets): the unit's packed records, its tile records, its
// restore_cols slice, the gathered x values (16 per tile) and its lane schedule.
constexpr uint32_t kOffStream = 0;
constexpr uint32_t kOffTiles = CB_B_MAX;
constexpr uint32_t kOffRcols = kOffTiles + CB_T_MAX * 16;
constexpr uint32_t kOffXs = kOffRcols + CB_RC_MAX * 4;
constexpr uint32_t kOffSched = kOffXs + CB_T_MAX * 16 * 8;
constexpr uint32_t kStageBytes = (kOffSched + CB_SCHED_MAX + 127) & ~127u;
static_assert(kOffStream % 16 == 0 && kOffTiles % 16 == 0 && kOffRcols % 16 == 0 && kOffXs % 16 == 0 &&
              kOffSched % 16 == 0, "bulk copy destinations must be 16-byte aligned");

struct Scratch {
  uint4 tinfo[CB_T_MAX];        // per tile: value base, coordinate base, x-row base (smem offsets)
  double srow[CB_R_MAX];        // row sums
  double cval[32];              // per-lane carry value
  int32_t crow[32];             // per-lane carry row (-1 none, -2 no chunks)
};

struct Shared {
  __align__(128) uint8_t stage[kStages][kStageBytes];
  uint64_t bar_tma[kStages];
  uint64_t bar_empty[kStages];
  Scratch scratch[kConsumers];
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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ void cp_async_8(uint32_t dst_smem, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst_smem), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t align16u(uint32_t v) { return (v + 15u) & ~15u; }

__device__ void set_error(const RunArgs& a, uint32_t code) { atomicOr(a.err, code); }

// ---- producer: one lane issues the bulk copies of every unit, in ticket order ------------
__device__ void producer(const RunArgs& a, Shared& sh, const uint32_t* list, uint32_t nu) {
  uint32_t issued = 0;
  bool ok = true;
  for (uint32_t j = 0; j < nu; ++j) {
    const uint32_t s = j % kStages, q = j / kStages;
    if (q > 0 && !mbar_wait(&sh.bar_empty[s], (q - 1) & 1)) { ok = false; break; }
    const CbUnit u = a.units[list[j]];
    uint8_t* S = sh.stage[s];
    mbar_arrive_expect_tx(&sh.bar_tma[s], u.nbytes + 16u * u.ntiles + 4u * u.rc_n + u.sched_bytes);
    if (u.nbytes) bulk_g2s(S + kOffStream, a.stream + (size_t)u.byte_lo16 * 16, u.nbytes, &sh.bar_tma[s]);
    if (u.ntiles) bulk_g2s(S + kOffTiles, a.tiles + u.tile_lo, 16u * u.ntiles, &sh.bar_tma[s]);
    if (u.rc_n) bulk_g2s(S + kOffRcols, a.rcols + u.rc_lo, 4u * u.rc_n, &sh.bar_tma[s]);
    if (u.sched_bytes) bulk_g2s(S + kOffSched, a.sched + (size_t)u.sched16 * 4, u.sched_bytes, &sh.bar_tma[s]);
    issued = j + 1;
  }
  if (!ok) {
    set_error(a, 1u);
    *(volatile uint32_t*)&sh.abort_flag = 1;
    // drain: the copies of the last kStages tickets may still be in flight
    for (uint32_t j = issued > (uint32_t)kStages ? issued - kStages : 0; j < issued; ++j)
      mbar_wait(&sh.bar_tma[j % kStages], (j / kStages) & 1);
  }
}

// ---- consumer -----------------------------------------------------------------------------
// sm: base of the CTA's shared memory; so: offset of the unit's stage in it.
__device__ void consume_unit(const RunArgs& a, const CbUnit& u, uint8_t* sm, uint32_t so, uint32_t ident_off,
                             Scratch& sc, int lane) {
  uint8_t* S = sm + so;
  const uint32_t T = u.ntiles;
  const uint32_t byte_lo = u.byte_lo16 * 16u;
  const int64_t row0 = (int64_t)u.brow_lo * CB_BLK;
  const int64_t rows_left = a.m - row0;
  const int64_t rows_unit = (int64_t)CB_BLK * u.nbr;
  const uint32_t R = (uint32_t)(rows_unit < rows_left ? rows_unit : rows_left);
  const CbTile* tiles = reinterpret_cast<const CbTile*>(S + kOffTiles);
  const int32_t* rcols = reinterpret_cast<const int32_t*>(S + kOffRcols);
  const uint32_t xs_smem = smem_u32(S + kOffXs);

  // 0. gather the unit's x values into the stage (asynchronous; waited for before the walk)
  const uint32_t nx = 16u * T;
  for (uint32_t idx = lane; idx < nx; idx += 32) {
    const uint32_t t = idx >> 4, c = idx & 15u;
    const uint32_t xb = tiles[t].xbase;
    const int64_t col = a.aggregated ? (int64_t)rcols[xb - u.rc_lo + c] : (int64_t)xb + c;
    const bool valid = col >= 0 && col < a.n;
    cp_async_8(xs_smem + 8u * idx, a.x + (valid ? col : 0), valid ? 8u : 0u);
  }
  // 1. per-tile bases (lane = tile) and zeroed row sums
  if ((uint32_t)lane < T) {
    const CbTile rec = tiles[lane];
    const uint32_t soff = so + rec.vp16 * 16u - byte_lo;
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
    sc.tinfo[lane] = make_uint4(vb, cb, so + kOffXs + 128u * lane, 0u);
  }
  for (uint32_t r = lane; r < R; r += 32) sc.srow[r] = 0.0;
  cp_async_wait_all();
  __syncwarp();   // x values and tile bases are visible to every lane

  // 2. the lane's chunks: up to CB_CHUNK entries of one (tile, row) piece per step
  const uint8_t* sched = S + kOffSched;
  const uint16_t* desc = reinterpret_cast<const uint16_t*>(sched + CB_SCHED_HDR(R));
  const uint32_t h = reinterpret_cast<const uint16_t*>(sched)[lane];
  uint32_t row = h & 0xffu;
  const bool hs = (h >> 8) & 1u;
  const uint32_t nch = h >> 9;
  const uint32_t steps = __reduce_max_sync(0xffffffffu, nch);
  double acc = 0.0;
  bool first = true, open = false;
  int32_t own_row = -1;
  double own_val = 0.0;
  for (uint32_t i = 0; i < steps; ++i) {
    const uint32_t d = desc[i * 32u + lane];
    if (d) {
      const uint32_t t = d & 31u, o = (d >> 5) & 255u, len = (d >> 13) & 3u;
      const uint4 ti = sc.tinfo[t];
      const uint32_t va = ti.x + 8u * o, ca = ti.y + o, xr = ti.z;
      const uint32_t b0 = sm[ca];
      const double v0 = *reinterpret_cast<const double*>(sm + va);
      uint32_t b1 = 0, b2 = 0;
      double v1 = 0.0, v2 = 0.0;
      if (len > 1) { b1 = sm[ca + 1]; v1 = *reinterpret_cast<const double*>(sm + va + 8u); }
      if (len > 2) { b2 = sm[ca + 2]; v2 = *reinterpret_cast<const double*>(sm + va + 16u); }
      const double x0 = *reinterpret_cast<const double*>(sm + xr + ((b0 >> 4) << 3));
      acc = fma(v0, x0, acc);
      if (len > 1) acc = fma(v1, *reinterpret_cast<const double*>(sm + xr + ((b1 >> 4) << 3)), acc);
      if (len > 2) acc = fma(v2, *reinterpret_cast<const double*>(sm + xr + ((b2 >> 4) << 3)), acc);
      open = true;
      if (d & 0x8000u) {   // the chunk ends its row
        if (first && hs) { own_row = (int32_t)row; own_val = acc; }
        else sc.srow[row] = acc;
        acc = 0.0;
        first = false;
        open = false;
        row = sched[64u + row];
      }
    }
  }
  sc.crow[lane] = nch == 0 ? -2 : (open ? (int32_t)row : -1);
  sc.cval[lane] = acc;
  __syncwarp();
  if (own_row >= 0) {
    double sum = own_val;
    for (int j = (int)lane - 1; j >= 0; --j) {
      const int32_t cr = sc.crow[j];
      if (cr == -2) continue;
      if (cr != own_row) break;
      sum += sc.cval[j];
    }
    sc.srow[own_row] = sum;
  }
  __syncwarp();

  // 3. outputs
  const double alpha = a.alpha, beta = a.beta;
  if (u.split < 0) {
    for (uint32_t r = lane; r < R; r += 32) {
      const int64_t gr = row0 + r;
      double v = sc.srow[r];
      if (!a.alpha_one) v = alpha * v;
      if (a.beta_nonzero) v = fma(beta, a.y[gr], v);
      a.y[gr] = v;
    }
  } else {
    double* part = a.partial + (size_t)u.slot * 16;
    if (lane < 16) part[lane] = (uint32_t)lane < R ? sc.srow[lane] : 0.0;
    __threadfence();
    __syncwarp();
    uint32_t last = 0;
    if (lane == 0) last = atomicAdd(&a.split_count[u.split], 1u) == (uint32_t)u.nparts - 1u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      if ((uint32_t)lane < R && lane < 16) {
        const double* base = a.partial + (size_t)(u.slot - u.part) * 16;
        double sum = 0.0;
        for (uint32_t p = 0; p < u.nparts; ++p) sum += __ldcg(base + p * 16 + lane);
        const int64_t gr = row0 + lane;
        double v = a.alpha_one ? sum : alpha * sum;
        if (a.beta_nonzero) v = fma(beta, a.y[gr], v);
        a.y[gr] = v;
      }
      if (lane == 0) a.split_count[u.split] = 0;   // ready for the next launch
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) spmv_f64_kernel(const RunArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t w0 = a.worker_off[blockIdx.x], w1 = a.worker_off[blockIdx.x + 1];
  const uint32_t* list = a.worker_units + w0;
  const uint32_t nu = w1 - w0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh.bar_tma[s], 1);
      mbar_init(&sh.bar_empty[s], 1);
    }
    sh.ticket = 0;
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (uint32_t i = threadIdx.x; i < 256u; i += blockDim.x) sh.ident[i] = (uint8_t)((i & 15u) << 4);
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) producer(a, sh, list, nu);
    return;
  }
  Scratch& sc = sh.scratch[warp - 1];
  for (;;) {
    uint32_t j = 0;
    if (lane == 0) j = atomicAdd(&sh.ticket, 1u);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= nu) break;
    const uint32_t s = j % kStages, q = j / kStages;
    const bool ok = mbar_wait(&sh.bar_tma[s], q & 1);
    if (!__all_sync(0xffffffffu, ok) || *(volatile uint32_t*)&sh.abort_flag) {
      if (lane == 0) set_error(a, 2u);
      break;
    }
    const CbUnit u = a.units[list[j]];
    consume_unit(a, u, smem_raw, (uint32_t)(sh.stage[s] - smem_raw), (uint32_t)(sh.ident - smem_raw), sc, lane);
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.bar_empty[s]);
  }
}

}  // namespace

size_t spmv_f64_smem_bytes() { return sizeof(Shared); }
int spmv_f64_threads() { return kThreads; }

cudaError_t launch_spmv_f64(const RunArgs& a, int grid, cudaStream_t stream) {
  static bool configured[64] = {false};
  const size_t smem = sizeof(Shared);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(spmv_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  spmv_f64_kernel<<<grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace cb
