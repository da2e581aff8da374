// Tensor-core product of a BF16-valued matrix with k right-hand sides (cbspmv_spmm):
// Y = alpha * A * X + beta * Y, X (n x k) and Y (m x k) row-major, FP32, k <= 32 per launch.
//
// With k vectors every 16x16 sub-block of Sec. 3.1 is a real contraction: its 16 columns
// of X (16 x k) are multiplied by the sub-block (16 x 16) into 16 x k partial rows, the
// shape of the tensor cores' mma.sync.m16n8k16 (A = the sub-block, B = 16 x 8 columns of X,
// C = 16 x 8 FP32). A warp walks a segment of one block row's sub-blocks:
//   * the sub-block's record (COO / CSR / Dense, Sec. 3.2-3.3.2) is expanded into a zeroed
//     16x16 BF16 tile in the warp's shared memory (Algorithm 4's zero fill) and loaded as the
//     A fragment with ldmatrix;
//   * the X rows of its 16 columns (through restore_cols when aggregated, the x preload of
//     Algorithms 3/4) are loaded straight into B-fragment registers. The MMA takes BF16
//     operands, X is FP32: each x is split exactly into three BF16 parts, h + m + l, with
//     |x - (h + m + l)| <= 2^-25 |x|, and the three partial products are accumulated in
//     FP32 (products of two BF16 numbers are exact in FP32), so the result keeps FP32-level
//     accuracy while the stored values stay BF16. The split is done once per x by a first
//     pass into a workspace of 8 bytes per x (h, m; l), not once per sub-block using it;
//   * the 16 x k accumulators stay in registers across the block row's sub-blocks; whole
//     block rows write Y once, block rows cut into segments store 16 x k partial sums that a
//     second kernel adds in segment order.
// Segments are taken longest first by an atomic ticket. Columns past the matrix read zero;
// like Dense zero fill, a non-finite x in a sub-block's column reaches the rows of that
// sub-block (results are specified for finite x).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cb_layout.h"
#include "cb_spmm.h"

namespace cb {
namespace {

constexpr int kWarps = 16;
constexpr uint32_t kTileBytes = 16 * 16 * 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// x = h + m + l exactly up to 2^-25 |x|: three round-to-nearest BF16 parts
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Splits X (n x k, FP32, row-major with leading dimension ldx) into the workspace: element
// (i, j) of the n x kpad result holds h | m << 16 and l of split3(x_ij), zero past k.
__global__ void __launch_bounds__(256) split_x_kernel(const SpmmArgs a) {
  const uint64_t total = (uint64_t)a.n * (uint64_t)a.kpad;
  const float* X = static_cast<const float*>(a.x);
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = e / (uint64_t)a.kpad;
    const int j = (int)(e % (uint64_t)a.kpad);
    uint2 q = make_uint2(0u, 0u);
    if (j < a.k) {
      __nv_bfloat16 h, m, l;
      split3(X[(int64_t)i * a.ldx + j], h, m, l);
      q = make_uint2(pack2(h, m), pack2(l, __float2bfloat16_rn(0.f)));
    }
    a.xs[e] = q;
  }
}

// Sub-blocks are taken in rounds of kB: the records, column indices and X values of a
// round's sub-blocks are loaded stage by stage for all of them before any is multiplied, so
// the three dependent memory latencies of a sub-block (record, restore_cols, X) are paid
// once per round instead of once per sub-block.
template <int kNB, int kB>
__global__ void __launch_bounds__(32 * kWarps) spmm_bf16_kernel(const SpmmArgs a) {
  __shared__ __align__(128) uint8_t tiles_smem[kWarps * kTileBytes];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* T = tiles_smem + warp * kTileBytes;
  const uint32_t g = lane >> 2, tig = lane & 3;     // MMA group and thread in group
  const int k = a.k;
  float* Y = static_cast<float*>(a.y);
  constexpr uint32_t kNoEntry = 0xffffffffu;
  for (;;) {
    uint32_t s = 0;
    if (lane == 0) s = atomicAdd(a.counter, 1u);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= a.nseg) break;
    const SpmmSeg seg = a.segs[s];
    float c[kNB][4];
#pragma unroll
    for (int nb = 0; nb < kNB; ++nb) c[nb][0] = c[nb][1] = c[nb][2] = c[nb][3] = 0.f;
    for (uint32_t t0 = 0; t0 < seg.ntiles; t0 += kB) {
      // 1. the round's sub-block records (lane b loads sub-block b's 16 bytes)
      uint4 tw = make_uint4(0u, 0u, 0u, 0u);
      if (lane < kB && t0 + lane < seg.ntiles) tw = __ldg(reinterpret_cast<const uint4*>(a.tiles + seg.tile_lo + t0 + lane));
      CbTile tr[kB];
      bool live[kB];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const uint32_t w0 = __shfl_sync(0xffffffffu, tw.x, b), w1 = __shfl_sync(0xffffffffu, tw.y, b);
        const uint32_t w2 = __shfl_sync(0xffffffffu, tw.z, b), w3 = __shfl_sync(0xffffffffu, tw.w, b);
        tr[b].vp16 = w0;
        tr[b].xbase = w1;
        tr[b].brow = w2;
        tr[b].nnz = (uint16_t)(w3 & 0xffffu);
        tr[b].fmt = (uint8_t)((w3 >> 16) & 0xffu);
        live[b] = t0 + b < seg.ntiles;
      }
      // 2. this lane's entries (COO / CSR: entry lane + 32 i as coordinate << 16 | value;
      //    Dense: its 16 bytes of the 512 value bytes) and its four column indices
      uint32_t pre[kB][4];
      int32_t col[kB][4];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const uint8_t* rec = a.stream + (size_t)tr[b].vp16 * 16;
        if (live[b] && tr[b].fmt == CB_FMT_DENSE) {
          const uint4 d = __ldg(reinterpret_cast<const uint4*>(rec + 32) + lane);
          pre[b][0] = d.x; pre[b][1] = d.y; pre[b][2] = d.z; pre[b][3] = d.w;
        } else {
          const uint32_t ib = tr[b].fmt == CB_FMT_CSR ? 17u : 0u;
          const uint32_t vb = (ib + tr[b].nnz + 15u) & ~15u;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t e = (uint32_t)lane + 32u * i;
            pre[b][i] = (live[b] && e < tr[b].nnz)
                            ? ((uint32_t)rec[ib + e] << 16) | *reinterpret_cast<const uint16_t*>(rec + vb + 2 * e)
                            : kNoEntry;
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t kr = 2 * tig + (i & 1) + 8 * (i >> 1);
          const int64_t cc = !live[b] ? -1
                             : a.aggregated ? (int64_t)__ldg(a.rcols + tr[b].xbase + kr) : (int64_t)tr[b].xbase + kr;
          col[b][i] = cc < a.n ? (int32_t)cc : -1;
        }
      }
      // 3. the split X values of this lane's B fragments (zero past k and past n)
      uint2 xv[kB][kNB][4];
#pragma unroll
      for (int b = 0; b < kB; ++b)
#pragma unroll
        for (int nb = 0; nb < kNB; ++nb) {
          const int j = nb * 8 + (int)g;
#pragma unroll
          for (int i = 0; i < 4; ++i)
            xv[b][nb][i] = col[b][i] >= 0 ? __ldg(a.xs + (int64_t)col[b][i] * a.kpad + j) : make_uint2(0u, 0u);
        }
      // 4. each sub-block: A as a zero-filled 16x16 BF16 tile, row-major, then the MMAs
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        if (!live[b]) continue;
        if (tr[b].fmt == CB_FMT_DENSE) {
          *reinterpret_cast<uint4*>(T + 16 * lane) = make_uint4(pre[b][0], pre[b][1], pre[b][2], pre[b][3]);
        } else {
          *reinterpret_cast<uint4*>(T + 16 * lane) = make_uint4(0u, 0u, 0u, 0u);
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (pre[b][i] != kNoEntry) {
              const uint32_t cb = pre[b][i] >> 16;
              *reinterpret_cast<uint16_t*>(T + 2 * ((cb & 15u) * 16 + (cb >> 4))) = (uint16_t)(pre[b][i] & 0xffffu);
            }
          }
          // entries past 128 (CSR records under thresholds above 128): read at use
          const uint32_t ib = tr[b].fmt == CB_FMT_CSR ? 17u : 0u;
          const uint32_t vb = (ib + tr[b].nnz + 15u) & ~15u;
          const uint8_t* rec = a.stream + (size_t)tr[b].vp16 * 16;
          for (uint32_t e = (uint32_t)lane + 128u; e < tr[b].nnz; e += 32) {
            const uint32_t cb = rec[ib + e];
            *reinterpret_cast<uint16_t*>(T + 2 * ((cb & 15u) * 16 + (cb >> 4))) =
                *reinterpret_cast<const uint16_t*>(rec + vb + 2 * e);
          }
        }
        __syncwarp();
        uint32_t af[4];
        {
          const uint32_t q = lane >> 3, r = (lane & 7) + 8 * (q & 1), cl = 8 * (q >> 1);
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                       : "=r"(af[0]), "=r"(af[1]), "=r"(af[2]), "=r"(af[3])
                       : "r"(smem_addr(T + 2 * (r * 16 + cl))));
        }
#pragma unroll
        for (int nb = 0; nb < kNB; ++nb) {
          const uint2* q = xv[b][nb];
          // smallest parts first; rows 2 tig, 2 tig + 1 (and + 8) pair up in the B fragment
          mma_bf16(c[nb], af, __byte_perm(q[0].y, q[1].y, 0x5410), __byte_perm(q[2].y, q[3].y, 0x5410));
          mma_bf16(c[nb], af, __byte_perm(q[0].x, q[1].x, 0x7632), __byte_perm(q[2].x, q[3].x, 0x7632));
          mma_bf16(c[nb], af, __byte_perm(q[0].x, q[1].x, 0x5410), __byte_perm(q[2].x, q[3].x, 0x5410));
        }
        __syncwarp();   // the tile buffer is rewritten by the next sub-block
      }
    }
    // C fragment: rows g and g + 8, columns 2 tig, 2 tig + 1 of each 8-column block
    const int64_t row0 = (int64_t)seg.brow * CB_BLK;
#pragma unroll
    for (int nb = 0; nb < kNB; ++nb)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = (int)g + 8 * (i >> 1);
        const int j = nb * 8 + 2 * (int)tig + (i & 1);
        if (j >= k) continue;
        if (seg.slot == 0xffffffffu) {
          const int64_t gr = row0 + r;
          if (gr < a.m) {
            float* yp = Y + gr * a.ldy + j;
            float v = c[nb][i];
            if (!a.alpha_one) v = a.alpha * v;
            if (a.beta_nonzero) v = fmaf(a.beta, *yp, v);
            *yp = v;
          }
        } else {
          a.partial[((size_t)seg.slot * 16 + r) * k + j] = c[nb][i];
        }
      }
  }
}

// Adds the segments of every cut block row in segment order and writes Y.
__global__ void __launch_bounds__(256) spmm_combine_kernel(const SpmmArgs a) {
  const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t per = 16ull * (uint64_t)a.k;
  const uint64_t sr = gid / per;
  if (sr >= a.nsplit) return;
  const uint32_t r = (uint32_t)((gid % per) / a.k), j = (uint32_t)(gid % a.k);
  const SpmmSplit sp = a.splits[sr];
  const int64_t gr = (int64_t)sp.brow * CB_BLK + r;
  if (gr >= a.m) return;
  const float* p = a.partial + ((size_t)sp.slot0 * 16 + r) * a.k + j;
  float sum = p[0];
  for (uint32_t q = 1; q < sp.nparts; ++q) sum += p[(size_t)q * 16 * a.k];
  float* yp = static_cast<float*>(a.y) + gr * a.ldy + j;
  float v = a.alpha_one ? sum : a.alpha * sum;
  if (a.beta_nonzero) v = fmaf(a.beta, *yp, v);
  *yp = v;
}

}  // namespace

cudaError_t launch_spmm_bf16(const SpmmArgs& a, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (a.n > 0) {
    const uint64_t total = (uint64_t)a.n * (uint64_t)a.kpad;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152ull * 32 ? (total + 255) / 256 : 152ull * 32);
    split_x_kernel<<<blocks, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int nb = (a.k + 7) / 8;
  switch (nb) {   // rounds of 4 sub-blocks, 2 at the widest (registers)
    case 1: spmm_bf16_kernel<1, 4><<<grid, 32 * kWarps, 0, s>>>(a); break;
    case 2: spmm_bf16_kernel<2, 4><<<grid, 32 * kWarps, 0, s>>>(a); break;
    case 3: spmm_bf16_kernel<3, 2><<<grid, 32 * kWarps, 0, s>>>(a); break;
    case 4: spmm_bf16_kernel<4, 2><<<grid, 32 * kWarps, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || a.nsplit == 0) return e;
  const uint64_t threads = (uint64_t)a.nsplit * 16 * (uint64_t)a.k;
  spmm_combine_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cb
