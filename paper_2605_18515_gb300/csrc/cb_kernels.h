// Launch interface of the run kernels (kernels.cu), used by the C ABI (capi.cu).
#ifndef CB_KERNELS_H_
#define CB_KERNELS_H_
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cbspmv.h"
#include "cb_layout.h"

namespace cb {

struct RunArgs {
  const uint8_t* stream;        // packed tile records
  const CbTile* tiles;          // per-tile records, matrix order
  const int32_t* rcols;         // restore_cols (+ padding); unused when plain
  const CbUnit* units;
  const uint8_t* blob;          // unit blobs: tile records, restore_cols slice, lane schedule
  const uint32_t* worker_units; // unit ids per persistent CTA
  const uint32_t* worker_off;   // grid + 1 offsets into worker_units
  const void* x;                // n values of the vector type (double for F64, else float)
  void* y;                      // m values of the vector type
  void* partial;                // partial sums of split block rows (16 per slot, vector type)
  const CbSplitRow* split_rows; // block rows cut into several units
  uint32_t n_split_rows;
  uint32_t n_split_wide;        // the last n_split_wide split rows have many parts
  uint32_t* err;                // device error word
  int64_t m, n;
  double alpha, beta;
  int aggregated;
  int alpha_one;                // alpha == 1: skip the scaling multiply
  int beta_nonzero;             // beta != 0: read y
  int value_dtype;              // cbspmv_dtype_t of the stored values
  int nvec;                     // vectors computed in one pass: 1, 2 or 4 (single product only)
  int64_t ldx, ldy;             // distance in elements between consecutive vectors of x and y
  long long wait_budget;        // clock64 cycles a bounded device wait may take before it gives up
  int stuck_wait;               // test hook: the first wait is on a barrier nothing arrives at
  // lane-stream layout (FP64; lanes = 1): these replace stream, units and blob
  int lanes;
  const CbLaneUnit* lunits;     // units in worker order
  const void* lvals;            // values in the storage type (layout in cb_layout.h)
  const uint64_t* lwords;       // entry words, 4 per uint64
  const int32_t* lgcols;        // gather lists
};

size_t spmv_smem_bytes();      // dynamic shared memory of the largest instantiation
int spmv_warps(int value_dtype);   // worker warps per CTA of the run kernel for a value type
// Launches the run kernel for a.value_dtype and a.nvec vectors and, when the matrix has
// block rows cut into several units, the kernel that adds their parts (two launches on
// `stream`; a.partial must hold 16 * nvec values per slot). ev: NULL, or three events
// recorded on `stream` before the run kernel, between the two launches and after the last.
cudaError_t launch_spmv(const RunArgs& a, int grid, cudaStream_t stream, cudaEvent_t* ev = nullptr);
// Launches the products of `count` problems of one value type with one run-kernel launch
// per 64 problems (plus one combine launch each when any has split block rows). The
// problems must not share a partial-sum buffer (that is, come from distinct handles) and
// must all have nvec 1, or all nvec 4 (record layout; partial sums of 16 x 4 per slot).
cudaError_t launch_spmv_batch(const RunArgs* a, int count, int grid, cudaStream_t stream);
// Sets every run-kernel instantiation's shared-memory limit on the current device (done
// lazily by the launches too; needed before a stream capture).
cudaError_t configure_kernels();
// Re-packs nnz new FP64 values (CSR order) into the packed stream at the recorded value
// slots, converted to the storage type dtype.
cudaError_t launch_repack(uint8_t* stream, const uint32_t* slot, const double* val, int64_t nnz, int dtype,
                          int grid, cudaStream_t s);

}  // namespace cb
#endif
