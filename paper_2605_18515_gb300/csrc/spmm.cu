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
//     accuracy while the stored values stay BF16;
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

template <int kNB>
__global__ void __launch_bounds__(32 * kWarps) spmm_bf16_kernel(const SpmmArgs a) {
  __shared__ __align__(128) uint8_t tiles_smem[kWarps * kTileBytes];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* T = tiles_smem + warp * kTileBytes;
  const uint32_t g = lane >> 2, tig = lane & 3;     // MMA group and thread in group
  const int k = a.k;
  const float* X = static_cast<const float*>(a.x);
  float* Y = static_cast<float*>(a.y);
  for (;;) {
    uint32_t s = 0;
    if (lane == 0) s = atomicAdd(a.counter, 1u);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= a.nseg) break;
    const SpmmSeg seg = a.segs[s];
    float c[kNB][4];
#pragma unroll
    for (int nb = 0; nb < kNB; ++nb) c[nb][0] = c[nb][1] = c[nb][2] = c[nb][3] = 0.f;
    for (uint32_t t = 0; t < seg.ntiles; ++t) {
      const CbTile tr = a.tiles[seg.tile_lo + t];
      const uint8_t* rec = a.stream + (size_t)tr.vp16 * 16;
      // A: the sub-block as a zero-filled 16x16 BF16 tile, row-major
      if (tr.fmt == CB_FMT_DENSE) {
        *reinterpret_cast<uint4*>(T + 16 * lane) = __ldg(reinterpret_cast<const uint4*>(rec + 32) + lane);
      } else {
        *reinterpret_cast<uint4*>(T + 16 * lane) = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        const uint32_t ib = tr.fmt == CB_FMT_CSR ? 17u : 0u;
        const uint32_t vb = (ib + tr.nnz + 15u) & ~15u;
        for (uint32_t e = lane; e < tr.nnz; e += 32) {
          const uint32_t cb = rec[ib + e];
          const uint16_t v = *reinterpret_cast<const uint16_t*>(rec + vb + 2 * e);
          *reinterpret_cast<uint16_t*>(T + 2 * ((cb & 15u) * 16 + (cb >> 4))) = v;
        }
      }
      __syncwarp();
      uint32_t af[4];
      {
        const uint32_t q = lane >> 3, r = (lane & 7) + 8 * (q & 1), col = 8 * (q >> 1);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(af[0]), "=r"(af[1]), "=r"(af[2]), "=r"(af[3])
                     : "r"(smem_addr(T + 2 * (r * 16 + col))));
      }
      // B: the X rows of this lane's four columns of the sub-block (k rows 2 tig, 2 tig + 1,
      // 2 tig + 8, 2 tig + 9 of the MMA), zero past the matrix
      int64_t col[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t kr = 2 * tig + (i & 1) + 8 * (i >> 1);
        int64_t cc = a.aggregated ? (int64_t)__ldg(a.rcols + tr.xbase + kr) : (int64_t)tr.xbase + kr;
        col[i] = cc < a.n ? cc : -1;
      }
#pragma unroll
      for (int nb = 0; nb < kNB; ++nb) {
        const int j = nb * 8 + (int)g;
        float xv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = (col[i] >= 0 && j < k) ? __ldg(X + col[i] * a.ldx + j) : 0.f;
        __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split3(xv[i], h[i], m[i], l[i]);
        // smallest parts first
        mma_bf16(c[nb], af, pack2(l[0], l[1]), pack2(l[2], l[3]));
        mma_bf16(c[nb], af, pack2(m[0], m[1]), pack2(m[2], m[3]));
        mma_bf16(c[nb], af, pack2(h[0], h[1]), pack2(h[2], h[3]));
      }
      __syncwarp();   // the tile buffer is rewritten by the next sub-block
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
  const int nb = (a.k + 7) / 8;
  switch (nb) {
    case 1: spmm_bf16_kernel<1><<<grid, 32 * kWarps, 0, s>>>(a); break;
    case 2: spmm_bf16_kernel<2><<<grid, 32 * kWarps, 0, s>>>(a); break;
    case 3: spmm_bf16_kernel<3><<<grid, 32 * kWarps, 0, s>>>(a); break;
    case 4: spmm_bf16_kernel<4><<<grid, 32 * kWarps, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || a.nsplit == 0) return e;
  const uint64_t threads = (uint64_t)a.nsplit * 16 * (uint64_t)a.k;
  spmm_combine_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace cb
