// Internal interface between capi.cu (which owns the handle layout) and noalloc.cu.
#ifndef CB_NOALLOC_H_
#define CB_NOALLOC_H_
#include <string>

#include "../../include/cbspmv.h"
#include "cb_kernels.h"
#include "cb_plan.h"

namespace cb {
struct NoallocView {
  int device;
  int grid;
  const Plan* plan;
  RunArgs args;   // the handle's device arrays; x, y and scratch are filled by the caller
};
// Fills *v from a valid handle; false for an invalid one.
bool noalloc_view(cbspmv_handle_t h, NoallocView* v);
// Sets the calling thread's message returned by cbspmv_last_error().
void set_last_error(const std::string& msg);
// The argument checks of cbspmv_run (valid device handle, x and y present, aligned to their
// element size and not overlapping); sets the message and returns the status on failure.
cbspmv_status_t check_product_args(cbspmv_handle_t h, const void* x, const void* y);
}  // namespace cb
#endif
