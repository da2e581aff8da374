// Launch interface of the tensor-core multi-vector product (spmm.cu), used by capi.cu.
#ifndef CB_SPMM_H_
#define CB_SPMM_H_
#include <cuda_runtime.h>
#include <stdint.h>

#include "cb_layout.h"

namespace cb {

// A run of consecutive sub-blocks of one block row, multiplied by one warp.
struct SpmmSeg {
  uint32_t tile_lo, ntiles;   // sub-blocks [tile_lo, tile_lo + ntiles) of the matrix order
  uint32_t brow;              // block row
  uint32_t slot;              // partial-sum slot (block rows cut into segments), else 0xffffffff
};
// A block row cut into nparts segments with consecutive slots slot0 ...
struct SpmmSplit {
  uint32_t brow, slot0, nparts, pad;
};

struct SpmmArgs {
  const uint8_t* stream;      // packed sub-block records (every record plain: no direct units)
  const CbTile* tiles;        // sub-block records, matrix order
  const int32_t* rcols;       // restore_cols (+ padding) when aggregated
  const SpmmSeg* segs;        // longest first
  uint32_t nseg;
  const SpmmSplit* splits;
  uint32_t nsplit;
  float* partial;             // 16 x k per slot
  uint32_t* counter;          // segment ticket (zeroed before each launch)
  const void* x;              // n x k FP32, row-major, leading dimension ldx
  uint2* xs;                  // workspace, n x kpad: each x split into BF16 parts h | m << 16, l
  int kpad;                   // k rounded up to 8
  void* y;                    // m x k FP32, row-major, leading dimension ldy
  int64_t m, n, ldx, ldy;
  int k;                      // 1..32
  float alpha, beta;
  int alpha_one, beta_nonzero, aggregated;
};

// Enqueues the product (one persistent launch, plus one launch that adds the segments of
// cut block rows) on stream s.
cudaError_t launch_spmm_bf16(const SpmmArgs& a, int grid, cudaStream_t s);

}  // namespace cb
#endif
