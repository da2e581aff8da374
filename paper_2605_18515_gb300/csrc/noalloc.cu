// cbspmv_run_noalloc: the product of cbspmv_run with no allocation of any kind.
//
// The run needs scratch memory for block rows that the analysis cut into several units:
// 16 partial sums per unit part, which a second kernel adds in part order.
// cbspmv_run takes that scratch from a buffer the handle allocated. This entry point takes
// it from one fixed array that lives in the library's device image instead, so the call
// itself never allocates: it is for callers that may not call cudaMalloc, cudaFree or
// any allocating routine when they run the product (code whose device memory is owned
// by another allocator, such as a framework's memory pool, and code on a latency-critical
// path where an allocation, which can synchronise the device, is not acceptable).
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// kNoallocBytes of it until the process exits. Host code cannot use its name as a device
// address, so the address is looked up once per device with cudaGetSymbolAddress (with
// that device current) and cached; the first call on each device does this set-up.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/cbspmv.h"
#include "cb_noalloc.h"

namespace {

constexpr size_t kNoallocMaxSlots = 63488;       // partial-sum slots (16 doubles each)
constexpr size_t kNoallocBytes = kNoallocMaxSlots * 16 * sizeof(double);   // 7.75 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" cbspmv_status_t cbspmv_run_noalloc(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta,
                                              void* stream) {
  cb::NoallocView v;
  if (!cb::noalloc_view(h, &v)) {
    cb::set_last_error("invalid handle");
    return CBSPMV_ERR_INVALID;
  }
  if (v.device < 0 || v.device >= kMaxDevices) {
    cb::set_last_error("cbspmv_run_noalloc needs a handle analysed for a device (0..63)");
    return CBSPMV_ERR_INVALID;
  }
  const cb::Plan& p = *v.plan;
  if ((size_t)p.n_slots > kNoallocMaxSlots) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "cbspmv_run_noalloc: matrix needs %d partial-sum slots; the static scratch holds at most %zu",
             p.n_slots, kNoallocMaxSlots);
    cb::set_last_error(buf);
    return CBSPMV_ERR_INVALID;
  }
  // the checks of cbspmv_run: x and y present, aligned to their element size, not overlapping
  const cbspmv_status_t chk = cb::check_product_args(h, x, y);
  if (chk != CBSPMV_OK) return chk;
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != v.device) e = cudaSetDevice(v.device);
  if (e != cudaSuccess) {
    cb::set_last_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return CBSPMV_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[v.device]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e == cudaSuccess) g_scratch_addr[v.device] = ptr;
    }
    base = g_scratch_addr[v.device];
  }
  cbspmv_status_t st = CBSPMV_OK;
  if (!base) {
    cb::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    st = CBSPMV_ERR_CUDA;
  } else if (p.m > 0) {
    // Every slot a run reads was written earlier in the same run, so the array's previous
    // contents never matter and nothing needs clearing.
    cb::RunArgs a = v.args;
    a.x = x;
    a.y = y;
    a.partial = base;
    a.alpha = alpha;
    a.beta = beta;
    a.alpha_one = alpha == 1.0;
    a.beta_nonzero = beta != 0.0;
    e = cb::launch_spmv(a, v.grid, (cudaStream_t)stream);
    if (e != cudaSuccess) {
      cb::set_last_error(std::string("cbspmv_run_noalloc: ") + cudaGetErrorString(e));
      st = CBSPMV_ERR_CUDA;
    }
  }
  if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
  if (st == CBSPMV_OK) cb::set_last_error("");
  return st;
}
