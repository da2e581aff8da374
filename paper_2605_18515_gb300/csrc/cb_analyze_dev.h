// Device-side analysis (analyze_dev.cu): the lane-stream layout built on the GPU from a CSR
// that lives on the device.
#ifndef CB_ANALYZE_DEV_H_
#define CB_ANALYZE_DEV_H_
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/cbspmv.h"
#include "cb_layout.h"
#include "cb_plan.h"

namespace cb {

// One chunk of a global-memory merge level: outputs [d0, d0 + chunk) of the stable merge of
// the runs [a0, a0 + la) and [a0 + la, a0 + la + lb).
struct MergeItem {
  int64_t a0;
  int32_t la, lb, d0, pad;
};

// Device arrays the device analysis leaves for the handle (allocated with the given
// allocator; owned by the caller on success, freed by analyze_device on failure).
struct DevLanes {
  CbLaneUnit* lunits = nullptr;
  uint8_t* lvals = nullptr;   // lvals_count values of the storage type
  uint64_t* lwords = nullptr;
  int32_t* lgcols = nullptr;
  int32_t* rcols = nullptr;    // restore_cols (+ CB_RC_PAD zeros) when aggregated, else nullptr
  uint32_t* vslot = nullptr;   // value map (keep_value_map)
  size_t lvals_count = 0, lwords_count = 0, lgcols_count = 0;
};

typedef cudaError_t (*DevAllocFn)(void** p, size_t bytes);

// Analyses the CSR A (row_ptr, col_idx and val device pointers on the current device) into
// the lane-stream layout on stream s: *plan gets everything the host analysis gives a
// lane-stream handle except the host copies of the lane arrays and of restore_cols (which
// stay on the device in *out). Requires the lane-stream layout: FP64 values with
// opts.record_layout 0, or any value type with opts.record_layout 2. Errors as
// cbspmv_analyze (CBSPMV_ERR_NOT_CANONICAL for an invalid CSR, found on the device before
// any other use of its arrays).
cbspmv_status_t analyze_device(const cbspmv_csr_t& A, const cbspmv_opts_t& opts, int n_workers, cudaStream_t s,
                               DevAllocFn alloc, Plan* plan, DevLanes* out, std::string* msg);

}  // namespace cb
#endif
