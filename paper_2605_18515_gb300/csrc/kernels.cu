// Run kernel of the blocked SpMV, y = alpha * A * x + beta * y, FP64, for sm_103a.
//
// The paper's kernel (Sec. 3.5, Algorithms 3 and 4) maps one sub-block to one warp,
// preloads x into shared memory (plain tiles) or reads it through restore_cols
// (aggregated tiles), reduces with warp shuffles and adds into y with atomics. On GB300
// the FP64 pipe is the scarce unit (a warp-wide DFMA occupies it for ~19 cycles per SM
// and lanes that are masked off cost the same), so this kernel keeps the data structure
// and the per-tile decoding of the paper but reorganises the work:
//
//   * Persistent grid, one CTA per SM: warp 0 is a producer, warps 1..CB_CONSUMERS are
//     consumers. The producer stages each unit of work (a run of consecutive tiles) into
//     a ring of CB_STAGES shared-memory stages with bulk TMA copies (cp.async.bulk) of the
//     unit's packed records, tile records and restore_cols slice, then gathers the
//     unit's x values into the stage with cp.async (the x preload of Algorithms 3/4, for
//     aggregated and plain tiles alike). mbarriers hand stages between the warps.
//   * A consumer builds per-tile row tables from the staged bytes (the CSR row pointer,
//     the COO coordinate bytes of Algorithm 3, the fixed rows of Algorithm 4), then
//     splits the unit's multiply-adds into 32 equal, contiguous runs of its row-major
//     entry order, one run per lane. Each lane walks its run with one DFMA per entry, so
//     every FP64 instruction is issued with all 32 lanes busy.
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
constexpr int kLag = 2;                       // producer gathers x for unit j - kLag
constexpr long long kWaitBudget = 4000000000LL;   // clock64 cycles (~2 s) per wait

struct Stage {
  uint8_t stream[CB_B_MAX];
  CbTile tiles[CB_T_MAX];
  int32_t rcols[CB_RC_MAX];
  double xs[CB_T_MAX * 16];
};
static_assert(sizeof(Stage) % 16 == 0, "stage alignment");

struct Scratch {
  uint8_t cnt[CB_T_MAX][16];    // entries of row r in tile t
  uint8_t st[CB_T_MAX][16];     // first entry of row r in tile t (COO/CSR) or 16r (Dense)
  uint32_t tinfo[CB_T_MAX][2];  // {value byte offset | index byte offset << 16, fmt | brl << 8}
  uint32_t tot[CB_R_MAX];       // entries per row of the unit
  uint16_t P[CB_R_MAX + 8];     // exclusive prefix of tot
  uint8_t tb_lo[CB_NBR_MAX], tb_hi[CB_NBR_MAX];
  double srow[CB_R_MAX];
  double cval[32];
  int32_t crow[32];
};

struct Shared {
  Stage stage[kStages];
  uint64_t bar_tma[kStages];
  uint64_t bar_full[kStages];
  uint64_t bar_empty[kStages];
  Scratch scratch[kConsumers];
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
__device__ __forceinline__ void cp_async_8(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t align16u(uint32_t v) { return (v + 15u) & ~15u; }

__device__ void set_error(const RunArgs& a, uint32_t code) { atomicOr(a.err, code); }

// ---- producer ---------------------------------------------------------------------------
__device__ void producer(const RunArgs& a, Shared& sh, const uint32_t* list, uint32_t nu, int lane) {
  uint32_t issued = 0;      // units whose bulk copies were issued
  uint32_t gathered = 0;    // units whose x gather was issued (their bulk data observed)
  bool ok = true;
  for (uint32_t j = 0; j < nu + kLag && ok; ++j) {
    if (j < nu) {
      const uint32_t s = j % kStages, q = j / kStages;
      if (q > 0 && !mbar_wait(&sh.bar_empty[s], (q - 1) & 1)) { ok = false; break; }
      if (lane == 0) {
        const CbUnit u = a.units[list[j]];
        const uint32_t bytes = u.nbytes + 16u * u.ntiles + 4u * u.rc_n;
        mbar_arrive_expect_tx(&sh.bar_tma[s], bytes);
        Stage& S = sh.stage[s];
        if (u.nbytes) bulk_g2s(S.stream, a.stream + (size_t)u.byte_lo16 * 16, u.nbytes, &sh.bar_tma[s]);
        if (u.ntiles) bulk_g2s(S.tiles, a.tiles + u.tile_lo, 16u * u.ntiles, &sh.bar_tma[s]);
        if (u.rc_n) bulk_g2s(S.rcols, a.rcols + u.rc_lo, 4u * u.rc_n, &sh.bar_tma[s]);
      }
      __syncwarp();
      issued = j + 1;
    }
    if (j >= (uint32_t)kLag) {
      const uint32_t jj = j - kLag;
      const uint32_t s = jj % kStages, q = jj / kStages;
      if (!mbar_wait(&sh.bar_tma[s], q & 1)) { ok = false; break; }
      gathered = jj + 1;
      const CbUnit u = a.units[list[jj]];
      Stage& S = sh.stage[s];
      const uint32_t nx = 16u * u.ntiles;
      for (uint32_t idx = lane; idx < nx; idx += 32) {
        const uint32_t t = idx >> 4, c = idx & 15u;
        const uint32_t xb = S.tiles[t].xbase;
        int64_t col = a.aggregated ? (int64_t)S.rcols[xb - u.rc_lo + c] : (int64_t)xb + c;
        const bool valid = col >= 0 && col < a.n;
        cp_async_8(&S.xs[idx], a.x + (valid ? col : 0), valid ? 8u : 0u);
      }
      cp_async_arrive_noinc(&sh.bar_full[s]);
    }
  }
  if (!ok) {
    if (lane == 0) set_error(a, 1u);
    sh.abort_flag = 1;
    // drain: bulk copies issued but not yet observed complete
    for (uint32_t jj = gathered; jj < issued; ++jj)
      mbar_wait(&sh.bar_tma[jj % kStages], (jj / kStages) & 1);
  }
  cp_async_wait_all();
}

// ---- consumer -----------------------------------------------------------------------------
__device__ void consume_unit(const RunArgs& a, const CbUnit& u, Stage& S, Scratch& sc, int lane) {
  const uint32_t T = u.ntiles;
  const uint32_t byte_lo = u.byte_lo16 * 16u;
  const int64_t row0 = (int64_t)u.brow_lo * CB_BLK;
  const int64_t rows_left = a.m - row0;
  const int64_t rows_unit = (int64_t)CB_BLK * u.nbr;
  const uint32_t R = (uint32_t)(rows_unit < rows_left ? rows_unit : rows_left);

  // init per-row totals, block-row tile ranges and row sums
  for (uint32_t r = lane; r < R; r += 32) { sc.tot[r] = 0; sc.srow[r] = 0.0; }
  if (lane < CB_NBR_MAX) { sc.tb_lo[lane] = 0; sc.tb_hi[lane] = 0; }
  __syncwarp();

  // 1. per-tile row tables, two tiles per iteration (one per half warp)
  const uint32_t half = lane >> 4, r = lane & 15u;
  for (uint32_t t0 = 0; t0 < T; t0 += 2) {
    const uint32_t t = t0 + half;
    uint32_t cnt = 0, st = 0;
    bool active = t < T;
    uint32_t fmt = 0, brl = 0;
    if (active) {
      const CbTile rec = S.tiles[t];
      const uint32_t soff = rec.vp16 * 16u - byte_lo;
      fmt = rec.fmt;
      brl = rec.brow - u.brow_lo;
      const uint32_t nnz = rec.nnz;
      uint32_t vb, ib;
      if (fmt == CB_FMT_CSR) {
        ib = soff + 17u;
        vb = soff + align16u(17u + nnz);
        st = S.stream[soff + r];
        cnt = S.stream[soff + r + 1] - st;
      } else if (fmt == CB_FMT_DENSE) {
        ib = 0;
        vb = soff + 32u;
        st = 16u * r;
        cnt = 16u;
      } else {
        ib = soff;
        vb = soff + align16u(nnz);
        // COO: entries sorted by row; lane r looks at entries r and r + 16. An entry that
        // starts a row records the start, an entry that ends a row records the end.
        st = 0;
        cnt = 0;
        sc.cnt[t][r] = 0;
        sc.st[t][r] = 0;
      }
      if (r == 0) {
        sc.tinfo[t][0] = vb | (ib << 16);
        sc.tinfo[t][1] = fmt | (brl << 8);
      }
    }
    __syncwarp();
    if (active && fmt == CB_FMT_COO) {
      const CbTile rec = S.tiles[t];
      const uint32_t soff = rec.vp16 * 16u - byte_lo;
      const uint32_t nnz = rec.nnz;
#pragma unroll
      for (uint32_t e = r; e < 32; e += 16) {
        if (e < nnz) {
          const uint32_t row = S.stream[soff + e] & 15u;
          const uint32_t prev = e > 0 ? (S.stream[soff + e - 1] & 15u) : 0xffu;
          const uint32_t next = e + 1 < nnz ? (S.stream[soff + e + 1] & 15u) : 0xffu;
          if (row != prev) sc.st[t][row] = (uint8_t)e;
          if (row != next) sc.cnt[t][row] = (uint8_t)(e + 1);   // end, fixed below
        }
      }
    }
    __syncwarp();
    if (active) {
      if (fmt == CB_FMT_COO) {
        const uint32_t end = sc.cnt[t][r];
        st = sc.st[t][r];
        cnt = end ? end - st : 0;
      }
      sc.cnt[t][r] = (uint8_t)cnt;
      sc.st[t][r] = (uint8_t)st;
      if (cnt) atomicAdd(&sc.tot[brl * 16u + r], cnt);
    }
    __syncwarp();
  }
  // 2. tile range of every block row in the unit
  for (uint32_t t = lane; t < T; t += 32) {
    const uint32_t b = sc.tinfo[t][1] >> 8;
    const uint32_t bp = t > 0 ? (sc.tinfo[t - 1][1] >> 8) : 0xffffu;
    const uint32_t bn = t + 1 < T ? (sc.tinfo[t + 1][1] >> 8) : 0xffffu;
    if (b != bp) sc.tb_lo[b] = (uint8_t)t;
    if (b != bn) sc.tb_hi[b] = (uint8_t)(t + 1);
  }
  // 3. exclusive prefix of row totals
  __syncwarp();
  uint32_t carry = 0;
  for (uint32_t base = 0; base < R; base += 32) {
    const uint32_t rr = base + lane;
    const uint32_t v = rr < R ? sc.tot[rr] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= (uint32_t)d) incl += o;
    }
    if (rr < R) sc.P[rr] = (uint16_t)(carry + incl - v);
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) sc.P[R] = (uint16_t)carry;
  __syncwarp();
  const uint32_t W = carry;

  // 4. this lane's contiguous run [lo, hi) of the row-major entry order
  const uint32_t lo = (uint32_t)(((uint64_t)lane * W) >> 5);
  const uint32_t hi = (uint32_t)(((uint64_t)(lane + 1) * W) >> 5);
  int32_t own_row = -1;
  double own_val = 0.0;
  int32_t carry_row = -1;
  double acc = 0.0;
  if (hi > lo) {
    // row containing position lo: largest r with P[r] <= lo
    uint32_t rlo = 0, rhi = R;   // P[rlo] <= lo < P[rhi]
    while (rhi - rlo > 1) {
      const uint32_t mid = (rlo + rhi) >> 1;
      if (sc.P[mid] <= lo) rlo = mid; else rhi = mid;
    }
    uint32_t row = rlo;
    uint32_t q = lo - sc.P[row];
    const bool head_shared = q > 0;
    uint32_t b = row >> 4, rr = row & 15u;
    uint32_t t = sc.tb_lo[b];
    while (q >= sc.cnt[t][rr]) { q -= sc.cnt[t][rr]; ++t; }
    uint32_t k = sc.st[t][rr] + q;
    uint32_t rem = sc.cnt[t][rr] - q;
    uint32_t ti0 = sc.tinfo[t][0], ti1 = sc.tinfo[t][1];
    uint32_t vb = ti0 & 0xffffu, ib = ti0 >> 16;
    bool dense = (ti1 & 0xffu) == CB_FMT_DENSE;
    const double* xs_t = &S.xs[t * 16];
    bool first = true, started = false;
    for (uint32_t i = lo; i < hi; ++i) {
      const uint32_t c = dense ? (k & 15u) : ((uint32_t)S.stream[ib + k] >> 4);
      const double v = *reinterpret_cast<const double*>(&S.stream[vb + 8u * k]);
      acc = fma(v, xs_t[c], acc);
      started = true;
      ++k;
      if (--rem == 0) {
        // next tile of this row inside the block row
        const uint32_t tend = sc.tb_hi[b];
        ++t;
        while (t < tend && sc.cnt[t][rr] == 0) ++t;
        if (t < tend) {
          k = sc.st[t][rr];
          rem = sc.cnt[t][rr];
        } else {
          // row complete
          if (first && head_shared) { own_row = (int32_t)row; own_val = acc; }
          else sc.srow[row] = acc;
          acc = 0.0;
          started = false;
          first = false;
          if (i + 1 < hi) {
            do { ++row; } while (sc.P[row + 1] == sc.P[row]);   // next row with entries
            b = row >> 4;
            rr = row & 15u;
            t = sc.tb_lo[b];
            while (sc.cnt[t][rr] == 0) ++t;
            k = sc.st[t][rr];
            rem = sc.cnt[t][rr];
          }
        }
        ti0 = sc.tinfo[t < CB_T_MAX ? t : 0][0];
        ti1 = sc.tinfo[t < CB_T_MAX ? t : 0][1];
        vb = ti0 & 0xffffu;
        ib = ti0 >> 16;
        dense = (ti1 & 0xffu) == CB_FMT_DENSE;
        xs_t = &S.xs[(t < CB_T_MAX ? t : 0) * 16];
      }
    }
    if (started) carry_row = (int32_t)row;
  }
  sc.crow[lane] = hi > lo ? carry_row : -2;     // -2: empty run, contributes nothing
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

  // 5. outputs
  const double alpha = a.alpha, beta = a.beta;
  if (u.split < 0) {
    for (uint32_t rr = lane; rr < R; rr += 32) {
      const int64_t gr = row0 + rr;
      double v = sc.srow[rr];
      if (!a.alpha_one) v = alpha * v;
      if (a.beta_nonzero) v = fma(beta, a.y[gr], v);
      a.y[gr] = v;
    }
  } else {
    double* part = a.partial + (size_t)u.slot * 16;
    if (lane < 16) part[lane] = sc.srow[lane < R ? lane : 0];
    __threadfence();
    __syncwarp();
    uint32_t last = 0;
    if (lane == 0) last = atomicAdd(&a.split_count[u.split], 1u) == (uint32_t)u.nparts - 1u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      if (lane < R && lane < 16) {
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
      mbar_init(&sh.bar_full[s], 32);
      mbar_init(&sh.bar_empty[s], 1);
    }
    sh.ticket = 0;
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    producer(a, sh, list, nu, lane);
    return;
  }
  Scratch& sc = sh.scratch[warp - 1];
  for (;;) {
    uint32_t j = 0;
    if (lane == 0) j = atomicAdd(&sh.ticket, 1u);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= nu) break;
    const uint32_t s = j % kStages, q = j / kStages;
    bool ok = mbar_wait(&sh.bar_full[s], q & 1);
    ok = ok && mbar_wait(&sh.bar_tma[s], q & 1);
    if (!__all_sync(0xffffffffu, ok) || *(volatile uint32_t*)&sh.abort_flag) {
      if (lane == 0) set_error(a, 2u);
      break;
    }
    const CbUnit u = a.units[list[j]];
    consume_unit(a, u, sh.stage[s], sc, lane);
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.bar_empty[s]);
  }
}

}  // namespace

size_t spmv_f64_smem_bytes() { return sizeof(Shared); }
int spmv_f64_threads() { return kThreads; }

cudaError_t launch_spmv_f64(const RunArgs& a, int grid, cudaStream_t stream) {
  static bool configured = false;
  const size_t smem = sizeof(Shared);
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(spmv_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  spmv_f64_kernel<<<grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace cb
