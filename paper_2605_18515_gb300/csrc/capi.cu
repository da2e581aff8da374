// The C ABI of include/cbspmv.h: argument checking, handle ownership, device uploads and
// kernel launches. All errors become status codes plus a thread-local message.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cbspmv.h"
#include "cb_kernels.h"
#include "cb_analyze_dev.h"
#include "cb_noalloc.h"
#include "cb_plan.h"
#include "cb_spmm.h"

namespace {

thread_local std::string g_err;

cbspmv_status_t fail(cbspmv_status_t s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

cbspmv_status_t ok() {
  g_err.clear();
  return CBSPMV_OK;
}

// Makes `dev` current for the lifetime of the object and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) {
      err = cudaSetDevice(dev);
      changed = err == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// Device allocations of the library go through dev_malloc. Fault injection for tests: when
// the environment variable CBSPMV_FAIL_ALLOC_AFTER holds N >= 0 at the start of
// cbspmv_analyze, that call's allocation number N (counting from 0) fails as out of memory.
thread_local long g_fail_alloc_after = -1;
cudaError_t dev_malloc(void** p, size_t bytes) {
  if (g_fail_alloc_after == 0) {
    g_fail_alloc_after = -1;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (g_fail_alloc_after > 0) --g_fail_alloc_after;
  return cudaMalloc(p, bytes);
}
long env_long(const char* name, long dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  const long r = std::strtol(v, &end, 10);
  return (end && *end == 0) ? r : dflt;
}

#define CB_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA,      \
                  "%s: %s", #call, cudaGetErrorString(e_));                                \
  } while (0)

}  // namespace

struct cbspmv_handle_s {
  uint32_t magic = 0xCB5B0001u;
  cb::Plan plan;
  int device = -1;
  int grid = 0;
  size_t stream_bytes = 0;
  uint8_t* d_stream = nullptr;
  CbTile* d_tiles = nullptr;
  int32_t* d_rcols = nullptr;
  CbUnit* d_units = nullptr;
  uint8_t* d_blob = nullptr;
  uint32_t* d_wunits = nullptr;
  uint32_t* d_woff = nullptr;
  void* d_partial = nullptr;
  CbSplitRow* d_split_rows = nullptr;
  uint32_t* d_err = nullptr;
  void* d_xstage = nullptr;
  void* d_ystage = nullptr;
  void* d_partial_multi = nullptr;   // partial sums of 4-vector passes (allocated on first use)
  uint32_t* d_vslot = nullptr;       // value slot per CSR entry (keep_value_map)
  double* d_valstage = nullptr;      // staging of host values for cbspmv_update_values
  // lane-stream layout (FP64 values)
  CbLaneUnit* d_lunits = nullptr;
  uint8_t* d_lvals = nullptr;        // lvals_count values of the storage type
  uint64_t* d_lwords = nullptr;
  int32_t* d_lgcols = nullptr;
  size_t lvals_count = 0, lwords_count = 0, lgcols_count = 0;
  // tensor-core multi-vector product (cbspmv_spmm), built on first use
  cb::SpmmSeg* d_spmm_segs = nullptr;
  cb::SpmmSplit* d_spmm_splits = nullptr;
  float* d_spmm_partial = nullptr;
  uint32_t* d_spmm_counter = nullptr;
  uint2* d_spmm_xs = nullptr;          // split X workspace (n x kpad), grown on demand
  size_t spmm_xs_cap = 0;
  uint32_t spmm_nseg = 0, spmm_nsplit = 0;
  bool spmm_ready = false;
  long long wait_budget = 4000000000LL;   // device wait budget of the record kernel (clock64 cycles)
  int stuck_wait = 0;                     // test hook (CBSPMV_TEST_STUCK_WAIT)
  // bytes of one x or y element: double for FP64 values, float for the reduced types
  size_t esize() const { return plan.value_dtype == CBSPMV_F64 ? 8 : 4; }

  void free_device() {
    if (device < 0) return;
    DeviceGuard g(device);
    cudaDeviceSynchronize();
    void* ptrs[] = {d_stream, d_tiles, d_rcols, d_units, d_blob, d_wunits, d_woff, d_partial, d_split_rows,
                    d_err, d_xstage, d_ystage, d_partial_multi, d_vslot, d_valstage,
                    d_lunits, d_lvals, d_lwords, d_lgcols,
                    d_spmm_segs, d_spmm_splits, d_spmm_partial, d_spmm_counter, d_spmm_xs};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    d_stream = nullptr;
    d_tiles = nullptr;
    d_rcols = nullptr;
    d_units = nullptr;
    d_blob = nullptr;
    d_wunits = nullptr;
    d_woff = nullptr;
    d_partial = nullptr;
    d_split_rows = nullptr;
    d_err = nullptr;
    d_xstage = nullptr;
    d_ystage = nullptr;
    d_partial_multi = nullptr;
    d_vslot = nullptr;
    d_valstage = nullptr;
    d_lunits = nullptr;
    d_lvals = nullptr;
    d_lwords = nullptr;
    d_lgcols = nullptr;
    d_spmm_segs = nullptr;
    d_spmm_splits = nullptr;
    d_spmm_partial = nullptr;
    d_spmm_counter = nullptr;
    d_spmm_xs = nullptr;
    spmm_xs_cap = 0;
    spmm_ready = false;
  }
};

static bool valid_handle(cbspmv_handle_t h) { return h && h->magic == 0xCB5B0001u; }

template <class T>
static cudaError_t upload(T** dst, const T* src, size_t count, cudaStream_t s) {
  size_t bytes = count * sizeof(T);
  cudaError_t e = dev_malloc((void**)dst, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  if (bytes) e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
  return e;
}

extern "C" {

cbspmv_status_t cbspmv_default_opts(cbspmv_opts_t* o) {
  if (!o) return fail(CBSPMV_ERR_INVALID, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->th0 = 0.15;
  o->th1 = 32;
  o->th2 = 128;
  o->col_agg = -1;
  o->value_dtype = CBSPMV_F64;
  o->unit_work = 0;
  o->load_balance = 1;
  o->device = 0;
  return ok();
}

// True when the device analysis builds the handle of a device CSR: the lane-stream layout on
// a device, and the three arrays in device memory of that device.
static bool device_analysis_applies(const cbspmv_csr_t& A, const cbspmv_opts_t& o) {
  const bool lanes = cb::uses_lanes(o);
  if (!A.on_device || o.device < 0 || !lanes) return false;
  const void* ptrs[3] = {A.row_ptr, A.col_idx, A.val};
  for (int i = 0; i < (A.nnz > 0 ? 3 : 1); ++i) {
    cudaPointerAttributes at{};
    if (!ptrs[i] || cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != o.device) return false;
  }
  return true;
}

cbspmv_status_t cbspmv_analyze(const cbspmv_csr_t* A, const cbspmv_opts_t* opts_in, void* stream,
                               cbspmv_handle_t* out) {
  if (!A || !out) return fail(CBSPMV_ERR_INVALID, "NULL argument");
  *out = nullptr;
  cbspmv_opts_t opts;
  if (opts_in) opts = *opts_in; else cbspmv_default_opts(&opts);
  const bool dev_analysis = device_analysis_applies(*A, opts);
  if (A->on_device && !dev_analysis) {
    // the record layouts are analysed on the host: copy the three arrays down, then analyse
    // the copy
    if (A->m < 0 || A->n < 0 || A->nnz < 0) return fail(CBSPMV_ERR_INVALID, "negative size");
    if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val))) return fail(CBSPMV_ERR_INVALID, "NULL CSR array");
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> va;
    try {
      rp.resize((size_t)A->m + 1);
      ci.resize((size_t)A->nnz);
      va.resize((size_t)A->nnz);
    } catch (const std::bad_alloc&) {
      return fail(CBSPMV_ERR_OOM, "host allocation failed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    CB_CUDA(cudaMemcpyAsync(rp.data(), A->row_ptr, rp.size() * 8, cudaMemcpyDeviceToHost, s));
    if (A->nnz) {
      CB_CUDA(cudaMemcpyAsync(ci.data(), A->col_idx, ci.size() * 4, cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaMemcpyAsync(va.data(), A->val, va.size() * 8, cudaMemcpyDeviceToHost, s));
    }
    CB_CUDA(cudaStreamSynchronize(s));
    cbspmv_csr_t H = *A;
    H.row_ptr = rp.data();
    H.col_idx = ci.data();
    H.val = va.data();
    H.on_device = 0;
    return cbspmv_analyze(&H, opts_in, stream, out);
  }
  g_fail_alloc_after = env_long("CBSPMV_FAIL_ALLOC_AFTER", -1);
  struct ResetFail {   // the injected failure applies to this call only
    ~ResetFail() { g_fail_alloc_after = -1; }
  } reset_fail;
  if (opts.unit_work < 0 || opts.unit_work > 16384)
    return fail(CBSPMV_ERR_INVALID, "unit_work must be in [0, 16384]");
  int grid = 1;
  if (opts.device >= 0) {
    int ndev = 0;
    CB_CUDA(cudaGetDeviceCount(&ndev));
    if (opts.device >= ndev) return fail(CBSPMV_ERR_INVALID, "device %d not present", opts.device);
    DeviceGuard g(opts.device);
    CB_CUDA(g.err);
    int sms = 0, smem_optin = 0;
    CB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, opts.device));
    CB_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, opts.device));
    if ((size_t)smem_optin < cb::spmv_smem_bytes())
      return fail(CBSPMV_ERR_UNSUPPORTED, "device has %d B of shared memory per block, kernel needs %zu",
                  smem_optin, cb::spmv_smem_bytes());
    grid = sms;
  } else if (opts.device != -1) {
    return fail(CBSPMV_ERR_INVALID, "device must be >= 0 or -1 (host only)");
  }
  cbspmv_handle_t h = new (std::nothrow) cbspmv_handle_s();
  if (!h) return fail(CBSPMV_ERR_OOM, "host allocation failed");
  std::string msg;
  cbspmv_status_t st;
  cb::DevLanes dl;
  try {
    if (dev_analysis) {
      DeviceGuard g(opts.device);
      st = g.err == cudaSuccess ? cb::analyze_device(*A, opts, grid, (cudaStream_t)stream, dev_malloc, &h->plan, &dl, &msg)
                                : CBSPMV_ERR_CUDA;
      if (g.err != cudaSuccess) msg = cudaGetErrorString(g.err);
    } else {
      st = cb::analyze_host(*A, opts, grid, &h->plan, &msg);
    }
  } catch (const std::bad_alloc&) {
    st = CBSPMV_ERR_OOM;
    msg = "host allocation failed during analysis";
  }
  if (st != CBSPMV_OK) {
    delete h;
    return fail(st, "%s", msg.c_str());
  }
  h->device = opts.device;
  h->grid = grid;
  {
    const long wb = env_long("CBSPMV_WAIT_BUDGET_CYCLES", 0);
    if (wb > 0) h->wait_budget = wb;
    h->stuck_wait = env_long("CBSPMV_TEST_STUCK_WAIT", 0) == 1 ? 1 : 0;
  }
  if (opts.device < 0) {
    *out = h;
    return ok();
  }
  DeviceGuard g(opts.device);
  cudaStream_t s = (cudaStream_t)stream;
  cb::Plan& p = h->plan;
  h->stream_bytes = p.stream.size();
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  if (dev_analysis) {
    // the lane stream, restore_cols and the value map were built on the device
    h->d_lunits = dl.lunits;
    h->d_lvals = dl.lvals;
    h->d_lwords = dl.lwords;
    h->d_lgcols = dl.lgcols;
    h->d_rcols = dl.rcols;
    h->d_vslot = dl.vslot;
    h->lvals_count = dl.lvals_count;
    h->lwords_count = dl.lwords_count;
    h->lgcols_count = dl.lgcols_count;
  } else if (p.lanes) {
    step(upload(&h->d_lunits, p.lane_units.data(), p.lane_units.size(), s));
    step(upload(&h->d_lvals, p.lane_vals.data(), p.lane_vals.size(), s));
    step(upload(&h->d_lwords, p.lane_words.data(), p.lane_words.size(), s));
    step(upload(&h->d_lgcols, p.lane_gcols.data(), p.lane_gcols.size(), s));
    h->lvals_count = p.n_lane_vals;
    h->lwords_count = p.lane_words.size();
    h->lgcols_count = p.lane_gcols.size();
  } else {
    step(upload(&h->d_stream, p.stream.data(), p.stream.size(), s));
    step(upload(&h->d_tiles, p.tiles.data(), p.tiles.size(), s));
    step(upload(&h->d_rcols, p.restore_cols.data(), p.restore_cols.size(), s));
    step(upload(&h->d_units, p.units.data(), p.units.size(), s));
    step(upload(&h->d_blob, p.blob.data(), p.blob.size(), s));
  }
  step(upload(&h->d_wunits, p.worker_units.data(), p.worker_units.size(), s));
  step(upload(&h->d_woff, p.worker_off.data(), p.worker_off.size(), s));
  if (e == cudaSuccess) e = dev_malloc(&h->d_partial, (size_t)(p.n_slots ? p.n_slots : 1) * 16 * h->esize());
  step(upload(&h->d_split_rows, p.split_rows.data(), p.split_rows.size(), s));
  if (!p.value_slot.empty()) step(upload(&h->d_vslot, p.value_slot.data(), p.value_slot.size(), s));
  if (e == cudaSuccess) e = dev_malloc((void**)&h->d_err, 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, 4, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    h->free_device();
    delete h;
    return fail(e == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA, "upload failed: %s",
                cudaGetErrorString(e));
  }
  // the packed stream (or the lane stream) and the value map now live on the device;
  // export reads them back
  cb::ByteBuf().swap(p.stream);
  std::vector<uint32_t>().swap(p.value_slot);
  decltype(p.lane_vals)().swap(p.lane_vals);
  decltype(p.lane_words)().swap(p.lane_words);
  decltype(p.lane_gcols)().swap(p.lane_gcols);
  *out = h;
  return ok();
}

static cb::RunArgs run_args(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta) {
  const cb::Plan& p = h->plan;
  cb::RunArgs a{};
  a.stream = h->d_stream;
  a.tiles = h->d_tiles;
  a.rcols = h->d_rcols;
  a.units = h->d_units;
  a.blob = h->d_blob;
  a.worker_units = h->d_wunits;
  a.worker_off = h->d_woff;
  a.x = x;
  a.y = y;
  a.partial = h->d_partial;
  a.split_rows = h->d_split_rows;
  a.n_split_rows = (uint32_t)p.split_rows.size();
  a.n_split_wide = (uint32_t)p.n_split_wide;
  a.err = h->d_err;
  a.m = p.m;
  a.n = p.n;
  a.alpha = alpha;
  a.beta = beta;
  a.aggregated = p.aggregated ? 1 : 0;
  a.alpha_one = alpha == 1.0;
  a.beta_nonzero = beta != 0.0;
  a.value_dtype = p.value_dtype;
  a.nvec = 1;
  a.ldx = p.n;
  a.ldy = p.m;
  a.lanes = p.lanes ? 1 : 0;
  a.lunits = h->d_lunits;
  a.lvals = h->d_lvals;
  a.lwords = h->d_lwords;
  a.lgcols = h->d_lgcols;
  a.wait_budget = h->wait_budget;
  a.stuck_wait = h->stuck_wait;
  return a;
}

static cbspmv_status_t run_device(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta,
                                  cudaStream_t s, cudaEvent_t* ev = nullptr) {
  if (h->plan.m == 0) return ok();
  CB_CUDA(cb::launch_spmv(run_args(h, x, y, alpha, beta), h->grid, s, ev));
  return ok();
}

// Checks of a run on k right-hand sides stored column by column: X holds n x k values with
// leading dimension ldx, Y m x k with ldy (k = 1: x and y). Returns CBSPMV_OK or fails.
static cbspmv_status_t check_run_args(cbspmv_handle_t h, int64_t k, const void* X, int64_t ldx, const void* Y,
                                      int64_t ldy) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  if (h->device < 0) return fail(CBSPMV_ERR_INVALID, "host-only handle cannot run");
  const int64_t m = h->plan.m, n = h->plan.n;
  if (k < 0) return fail(CBSPMV_ERR_INVALID, "k must be >= 0");
  if (ldx < n || ldy < m) return fail(CBSPMV_ERR_INVALID, "leading dimensions must be >= n (X) and >= m (Y)");
  if (k == 0) return ok();
  if ((!X && n > 0) || (!Y && m > 0)) return fail(CBSPMV_ERR_INVALID, "NULL x or y");
  const int64_t es = (int64_t)h->esize();
  if (((uintptr_t)X & (es - 1)) || ((uintptr_t)Y & (es - 1)))
    return fail(CBSPMV_ERR_INVALID, "x and y must be aligned to their element size (%d bytes)", (int)es);
  if (X && Y && n > 0 && m > 0) {
    const char* xb = (const char*)X;
    const char* yb = (const char*)Y;
    const int64_t xspan = es * (ldx * (k - 1) + n), yspan = es * (ldy * (k - 1) + m);
    if (xb < yb + yspan && yb < xb + xspan) return fail(CBSPMV_ERR_INVALID, "x and y overlap");
  }
  return ok();
}

cbspmv_status_t cbspmv_run(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta, void* stream) {
  cbspmv_status_t st = check_run_args(h, 1, x, h && valid_handle(h) ? h->plan.n : 0, y,
                                      h && valid_handle(h) ? h->plan.m : 0);
  if (st != CBSPMV_OK) return st;
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  return run_device(h, x, y, alpha, beta, (cudaStream_t)stream);
}

cbspmv_status_t cbspmv_time_kernels(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta, int reps,
                                    void* stream, double* ms_main, double* ms_combine, int* launches_per_run) {
  cbspmv_status_t st = check_run_args(h, 1, x, h && valid_handle(h) ? h->plan.n : 0, y,
                                      h && valid_handle(h) ? h->plan.m : 0);
  if (st != CBSPMV_OK) return st;
  if (reps < 1 || reps > 100000) return fail(CBSPMV_ERR_INVALID, "reps must be in [1, 100000]");
  if (!ms_main || !ms_combine || !launches_per_run) return fail(CBSPMV_ERR_INVALID, "NULL output");
  *ms_main = *ms_combine = 0.0;
  {
    const cb::Plan& pl = h->plan;
    const int narrow = (int)pl.split_rows.size() - pl.n_split_wide;
    *launches_per_run = pl.m == 0 ? 0 : 1 + (narrow > 0 ? 1 : 0) + (pl.n_split_wide > 0 ? 1 : 0);
  }
  if (h->plan.m == 0) return ok();
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  cudaStream_t s = (cudaStream_t)stream;
  // events of up to kBatch runs are outstanding at a time; each batch is read back at its end
  constexpr int kBatch = 256;
  std::vector<cudaEvent_t> ev(3 * kBatch, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& v : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&v);
  double t_main = 0.0, t_comb = 0.0;
  for (int done = 0; e == cudaSuccess && done < reps;) {
    const int nb = reps - done < kBatch ? reps - done : kBatch;
    for (int i = 0; i < nb && st == CBSPMV_OK; ++i)
      st = run_device(h, x, y, alpha, beta, s, &ev[3 * i]);
    if (st != CBSPMV_OK) break;
    e = cudaStreamSynchronize(s);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
      float a = 0.f, b = 0.f;
      e = cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]);
      t_main += a;
      t_comb += b;
    }
    done += nb;
  }
  for (auto& v : ev)
    if (v) cudaEventDestroy(v);
  if (st != CBSPMV_OK) return st;
  if (e != cudaSuccess) return fail(CBSPMV_ERR_CUDA, "event timing failed: %s", cudaGetErrorString(e));
  *ms_main = t_main / reps;
  *ms_combine = h->plan.split_rows.empty() ? 0.0 : t_comb / reps;
  return ok();
}

// The partial-sum buffer of 4-vector passes (16 x 4 values per slot), allocated on first use.
static cbspmv_status_t ensure_partial_multi(cbspmv_handle_t h) {
  if (!h->d_partial_multi)
    CB_CUDA(dev_malloc(&h->d_partial_multi, (size_t)(h->plan.n_slots ? h->plan.n_slots : 1) * 16 * 4 * h->esize()));
  return ok();
}

// Whether cbspmv_run_multi computes several vectors per pass. FP64 lane streams: no, the
// FP64 FMA pipe bounds the product (passes of 1, 2 and 4 vectors measured 0.198, 0.236 and
// 0.295 ms per vector on the FEM band). Lane streams of the reduced types: yes, except for
// large matrices whose gathered x slots serve fewer than two stored entries each: a pass
// over four vectors gathers four values per slot, which on R-MAT scale 21 (about one entry
// per slot) measured slower per vector than single passes (0.189 against 0.148 ms, FP32),
// on the FEM band faster (0.093 against 0.116 ms, BF16); on small matrices the launches
// saved outweigh the gathers. The record layout: yes.
static bool multi_vector_passes(const cb::Plan& p) {
  if (!p.lanes) return true;
  if (p.vsize == 8) return false;
  return p.nnz < (int64_t{1} << 22) || 32 * (uint64_t)p.tiles.size() <= (uint64_t)p.nnz;
}

cbspmv_status_t cbspmv_run_multi(cbspmv_handle_t h, int k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                                 double alpha, double beta, void* stream) {
  cbspmv_status_t st = check_run_args(h, k, X, ldx, Y, ldy);
  if (st != CBSPMV_OK || k == 0) return st;
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  if (h->plan.m == 0) return ok();
  const cb::Plan& p = h->plan;
  const size_t es = h->esize();
  if (k > 1) {
    const cbspmv_status_t st = ensure_partial_multi(h);
    if (st != CBSPMV_OK) return st;
  }
  // passes of 4, then 2, then 1 vectors (records), of 4 then 1 (lane streams), or single
  // vectors (see multi_vector_passes); each pass reads the matrix once
  const bool multi = multi_vector_passes(p);
  for (int j = 0; j < k;) {
    const int nv = !multi ? 1 : k - j >= 4 ? 4 : p.lanes ? 1 : k - j >= 2 ? 2 : 1;
    cb::RunArgs a = run_args(h, (const char*)X + es * j * ldx, (char*)Y + es * j * ldy, alpha, beta);
    a.nvec = nv;
    a.ldx = ldx;
    a.ldy = ldy;
    if (nv > 1) a.partial = h->d_partial_multi;
    CB_CUDA(cb::launch_spmv(a, h->grid, (cudaStream_t)stream));
    j += nv;
  }
  return ok();
}

// Segments of the tensor-core product: every block row's sub-blocks in runs of at most
// kSpmmSegTiles (block rows without sub-blocks still get a segment, which writes their y),
// longest first; block rows cut into several segments get consecutive partial-sum slots.
static constexpr uint32_t kSpmmSegTiles = 64;
static cbspmv_status_t spmm_prepare(cbspmv_handle_t h, cudaStream_t s) {
  const cb::Plan& p = h->plan;
  std::vector<cb::SpmmSeg> segs;
  std::vector<cb::SpmmSplit> splits;
  uint32_t slot = 0;
  size_t t = 0;
  for (int64_t b = 0; b < p.nbr; ++b) {
    const size_t t0 = t;
    while (t < p.tiles.size() && p.tiles[t].brow == (uint32_t)b) ++t;
    const uint32_t T = (uint32_t)(t - t0);
    const uint32_t parts = T <= kSpmmSegTiles ? 1u : (T + kSpmmSegTiles - 1) / kSpmmSegTiles;
    if (parts > 1) splits.push_back({(uint32_t)b, slot, parts, 0u});
    for (uint32_t q = 0; q < parts; ++q) {
      const uint32_t lo = (uint32_t)t0 + q * kSpmmSegTiles;
      const uint32_t n = std::min<uint32_t>(kSpmmSegTiles, (uint32_t)t - lo);
      segs.push_back({lo, parts > 1 ? n : T, (uint32_t)b, parts > 1 ? slot++ : 0xffffffffu});
    }
  }
  std::stable_sort(segs.begin(), segs.end(),
                   [](const cb::SpmmSeg& x, const cb::SpmmSeg& y) { return x.ntiles > y.ntiles; });
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  step(upload(&h->d_spmm_segs, segs.data(), segs.size(), s));
  step(upload(&h->d_spmm_splits, splits.data(), splits.size(), s));
  if (e == cudaSuccess) e = dev_malloc((void**)&h->d_spmm_partial, (size_t)(slot ? slot : 1) * 16 * 32 * sizeof(float));
  if (e == cudaSuccess) e = dev_malloc((void**)&h->d_spmm_counter, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    void* ptrs[] = {h->d_spmm_segs, h->d_spmm_splits, h->d_spmm_partial, h->d_spmm_counter};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    h->d_spmm_segs = nullptr;
    h->d_spmm_splits = nullptr;
    h->d_spmm_partial = nullptr;
    h->d_spmm_counter = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA, "cbspmv_spmm set-up: %s",
                cudaGetErrorString(e));
  }
  h->spmm_nseg = (uint32_t)segs.size();
  h->spmm_nsplit = (uint32_t)splits.size();
  h->spmm_ready = true;
  return ok();
}

cbspmv_status_t cbspmv_spmm(cbspmv_handle_t h, int k, const void* X, int64_t ldx, void* Y, int64_t ldy,
                            double alpha, double beta, void* stream) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  if (h->device < 0) return fail(CBSPMV_ERR_INVALID, "host-only handle cannot run");
  const cb::Plan& p = h->plan;
  if (k < 0) return fail(CBSPMV_ERR_INVALID, "k must be >= 0");
  if (ldx < k || ldy < k) return fail(CBSPMV_ERR_INVALID, "leading dimensions must be >= k");
  if (k == 0 || p.m == 0) return ok();
  if (p.value_dtype != CBSPMV_BF16)
    return fail(CBSPMV_ERR_UNSUPPORTED, "cbspmv_spmm needs BF16 values (tensor-core path); use cbspmv_run_multi");
  if (p.lanes || p.stats.n_direct_units != 0)
    return fail(CBSPMV_ERR_UNSUPPORTED,
                "cbspmv_spmm needs the record layout with opts.plain_records = 1 (not the lane-stream layout)");
  if ((!X && p.n > 0) || !Y) return fail(CBSPMV_ERR_INVALID, "NULL X or Y");
  if (((uintptr_t)X & 3) || ((uintptr_t)Y & 3)) return fail(CBSPMV_ERR_INVALID, "X and Y must be 4-byte aligned");
  if (X && p.n > 0) {
    const char* xb = (const char*)X;
    const char* yb = (const char*)Y;
    const int64_t xspan = 4 * ((p.n - 1) * ldx + k), yspan = 4 * ((p.m - 1) * ldy + k);
    if (xb < yb + yspan && yb < xb + xspan) return fail(CBSPMV_ERR_INVALID, "X and Y overlap");
  }
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  cudaStream_t s = (cudaStream_t)stream;
  if (!h->spmm_ready) {
    const cbspmv_status_t st = spmm_prepare(h, s);
    if (st != CBSPMV_OK) return st;
  }
  // the workspace of the split X: n x kpad (k rounded up to 8, at most 32) elements of 8 bytes
  {
    const int kmax = k < 32 ? k : 32;
    const size_t need = (size_t)(p.n > 0 ? p.n : 1) * (size_t)((kmax + 7) / 8 * 8);
    if (need > h->spmm_xs_cap) {
      if (h->d_spmm_xs) {
        CB_CUDA(cudaStreamSynchronize(s));   // (earlier launches may still read it)
        cudaFree(h->d_spmm_xs);
        h->d_spmm_xs = nullptr;
        h->spmm_xs_cap = 0;
      }
      const cudaError_t e = dev_malloc((void**)&h->d_spmm_xs, need * sizeof(uint2));
      if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? CBSPMV_ERR_OOM : CBSPMV_ERR_CUDA, "cbspmv_spmm workspace: %s",
                    cudaGetErrorString(e));
      h->spmm_xs_cap = need;
    }
  }
  // 32 columns per launch (the 16 x 32 accumulators of a segment stay in registers)
  for (int j0 = 0; j0 < k; j0 += 32) {
    cb::SpmmArgs a{};
    a.stream = h->d_stream;
    a.tiles = h->d_tiles;
    a.rcols = h->d_rcols;
    a.segs = h->d_spmm_segs;
    a.nseg = h->spmm_nseg;
    a.splits = h->d_spmm_splits;
    a.nsplit = h->spmm_nsplit;
    a.partial = h->d_spmm_partial;
    a.counter = h->d_spmm_counter;
    a.x = (const float*)X + j0;
    a.y = (float*)Y + j0;
    a.m = p.m;
    a.n = p.n;
    a.ldx = ldx;
    a.ldy = ldy;
    a.k = k - j0 < 32 ? k - j0 : 32;
    a.xs = h->d_spmm_xs;
    a.kpad = (a.k + 7) / 8 * 8;
    a.alpha = (float)alpha;
    a.beta = (float)beta;
    a.alpha_one = alpha == 1.0;
    a.beta_nonzero = beta != 0.0;
    a.aggregated = p.aggregated ? 1 : 0;
    CB_CUDA(cb::launch_spmm_bf16(a, h->grid, s));
  }
  return ok();
}

cbspmv_status_t cbspmv_analyze_batched(int count, const cbspmv_csr_t* A, const cbspmv_opts_t* opts, void* stream,
                                       cbspmv_handle_t* out) {
  if (count < 0) return fail(CBSPMV_ERR_INVALID, "count must be >= 0");
  if (count == 0) return ok();
  if (!A || !out) return fail(CBSPMV_ERR_INVALID, "NULL argument");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  for (int i = 0; i < count; ++i) {
    cbspmv_status_t st = cbspmv_analyze(&A[i], opts, stream, &out[i]);
    if (st != CBSPMV_OK) {
      std::string msg = g_err;
      for (int j = 0; j < i; ++j) {
        cbspmv_destroy(out[j]);
        out[j] = nullptr;
      }
      return fail(st, "matrix %d: %s", i, msg.c_str());
    }
  }
  return ok();
}

cbspmv_status_t cbspmv_run_batched(int count, const cbspmv_handle_t* hs, const int* k, const void* const* X,
                                   void* const* Y, const double* alpha, const double* beta, void* stream) {
  if (count < 0) return fail(CBSPMV_ERR_INVALID, "count must be >= 0");
  if (count == 0) return ok();
  if (!hs || !X || !Y || !alpha || !beta) return fail(CBSPMV_ERR_INVALID, "NULL argument");
  // check every problem before enqueuing any work
  for (int i = 0; i < count; ++i) {
    const int ki = k ? k[i] : 1;
    cbspmv_handle_t h = hs[i];
    const bool v = valid_handle(h);
    cbspmv_status_t st = check_run_args(h, ki, X[i], v ? h->plan.n : 0, Y[i], v ? h->plan.m : 0);
    if (st != CBSPMV_OK) return fail(st, "problem %d: %s", i, std::string(g_err).c_str());
  }
  // One launch per (value type, round): round r holds the r-th product of every handle, so
  // no handle's partial-sum buffer is used twice within a launch.
  for (int i = 1; i < count; ++i)
    if (hs[i]->device != hs[0]->device) return fail(CBSPMV_ERR_INVALID, "problems on different devices");
  // Handles other than FP64 lane streams take their columns in passes of four where they
  // can (round r4 of quads holds the r4-th group of four columns of every such handle), the
  // rest one at a time (a batch of many matrices gains more from fewer launches than a
  // large R-MAT loses to the gathers of four vectors); the quads use each handle's 4-vector
  // partial-sum buffer, allocated here first.
  std::vector<std::vector<cb::RunArgs>> rounds;   // per round, all value types mixed
  std::vector<std::vector<cb::RunArgs>> quads;
  std::vector<std::pair<cbspmv_handle_t, int>> seen, seen4;
  auto occupancy = [](std::vector<std::pair<cbspmv_handle_t, int>>& v, cbspmv_handle_t h, int add) {
    for (auto& sh : v)
      if (sh.first == h) { const int o = sh.second; sh.second += add; return o; }
    v.push_back({h, add});
    return 0;
  };
  for (int i = 0; i < count; ++i) {
    cbspmv_handle_t h = hs[i];
    if (h->plan.m == 0) continue;
    const int ki = k ? k[i] : 1;
    const size_t es = h->esize();
    const int nq = h->plan.lanes && h->plan.vsize == 8 ? 0 : ki / 4;
    const int occ4 = occupancy(seen4, h, nq);
    for (int q = 0; q < nq; ++q) {
      if ((int)quads.size() <= occ4 + q) quads.resize(occ4 + q + 1);
      cb::RunArgs a = run_args(h, (const char*)X[i] + es * 4 * q * h->plan.n, (char*)Y[i] + es * 4 * q * h->plan.m,
                               alpha[i], beta[i]);
      a.nvec = 4;
      quads[occ4 + q].push_back(a);
    }
    const int occ = occupancy(seen, h, ki - 4 * nq);
    for (int j = 4 * nq; j < ki; ++j) {
      const int r = occ + j - 4 * nq;
      if ((int)rounds.size() <= r) rounds.resize(r + 1);
      rounds[r].push_back(run_args(h, (const char*)X[i] + es * j * h->plan.n, (char*)Y[i] + es * j * h->plan.m,
                                   alpha[i], beta[i]));
    }
  }
  if (rounds.empty() && quads.empty()) return ok();
  DeviceGuard g(hs[0]->device);
  CB_CUDA(g.err);
  for (auto& sh : seen4)
    if (sh.second > 0) {
      cbspmv_status_t st = ensure_partial_multi(sh.first);
      if (st != CBSPMV_OK) return st;
    }
  for (auto& rd : quads) {
    for (auto& a : rd) {
      for (auto& sh : seen4)
        if (sh.first->d_partial == a.partial) a.partial = sh.first->d_partial_multi;
    }
    for (int dt = CBSPMV_F64; dt <= CBSPMV_F16; ++dt) {
      std::vector<cb::RunArgs> sel;
      for (auto& a : rd)
        if (a.value_dtype == dt) sel.push_back(a);
      if (!sel.empty()) CB_CUDA(cb::launch_spmv_batch(sel.data(), (int)sel.size(), hs[0]->grid, (cudaStream_t)stream));
    }
  }
  for (auto& rd : rounds) {
    for (int dt = CBSPMV_F64; dt <= CBSPMV_F16; ++dt) {
      std::vector<cb::RunArgs> sel;
      for (auto& a : rd)
        if (a.value_dtype == dt) sel.push_back(a);
      if (!sel.empty()) CB_CUDA(cb::launch_spmv_batch(sel.data(), (int)sel.size(), hs[0]->grid, (cudaStream_t)stream));
    }
  }
  return ok();
}

cbspmv_status_t cbspmv_run_host(cbspmv_handle_t h, const void* x_host, void* y_host, double alpha, double beta,
                                void* stream) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  if (h->device < 0) return fail(CBSPMV_ERR_INVALID, "host-only handle cannot run");
  const cb::Plan& p = h->plan;
  if ((!x_host && p.n > 0) || (!y_host && p.m > 0)) return fail(CBSPMV_ERR_INVALID, "NULL x or y");
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t es = h->esize();
  if (!h->d_xstage) CB_CUDA(dev_malloc(&h->d_xstage, (size_t)(p.n ? p.n : 1) * es));
  if (!h->d_ystage) CB_CUDA(dev_malloc(&h->d_ystage, (size_t)(p.m ? p.m : 1) * es));
  if (p.n) CB_CUDA(cudaMemcpyAsync(h->d_xstage, x_host, (size_t)p.n * es, cudaMemcpyHostToDevice, s));
  if (beta != 0.0 && p.m) CB_CUDA(cudaMemcpyAsync(h->d_ystage, y_host, (size_t)p.m * es, cudaMemcpyHostToDevice, s));
  cbspmv_status_t st = run_device(h, h->d_xstage, h->d_ystage, alpha, beta, s);
  if (st != CBSPMV_OK) return st;
  if (p.m) CB_CUDA(cudaMemcpyAsync(y_host, h->d_ystage, (size_t)p.m * es, cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  return ok();
}

cbspmv_status_t cbspmv_update_values(cbspmv_handle_t h, const double* val, int on_device, void* stream) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  if (h->device < 0) return fail(CBSPMV_ERR_INVALID, "host-only handle");
  const cb::Plan& p = h->plan;
  if (!h->d_vslot) return fail(CBSPMV_ERR_INVALID, "the handle was analysed without keep_value_map");
  if (p.nnz == 0) return ok();
  if (!val) return fail(CBSPMV_ERR_INVALID, "NULL values");
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  cudaStream_t s = (cudaStream_t)stream;
  const double* dval = val;
  if (!on_device) {
    if (!h->d_valstage) CB_CUDA(dev_malloc((void**)&h->d_valstage, (size_t)p.nnz * 8));
    CB_CUDA(cudaMemcpyAsync(h->d_valstage, val, (size_t)p.nnz * 8, cudaMemcpyHostToDevice, s));
    dval = h->d_valstage;
  }
  uint8_t* dst = p.lanes ? h->d_lvals : h->d_stream;
  CB_CUDA(cb::launch_repack(dst, h->d_vslot, dval, p.nnz, p.value_dtype, h->grid, s));
  return ok();
}

cbspmv_status_t cbspmv_check_device(cbspmv_handle_t h, void* stream) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  if (h->device < 0) return ok();
  DeviceGuard g(h->device);
  CB_CUDA(g.err);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t err = 0;
  CB_CUDA(cudaStreamSynchronize(s));
  CB_CUDA(cudaMemcpy(&err, h->d_err, 4, cudaMemcpyDeviceToHost));
  if (err) {
    CB_CUDA(cudaMemset(h->d_err, 0, 4));
    return fail(CBSPMV_ERR_TIMEOUT, "a bounded device wait gave up (code 0x%x)", err);
  }
  return ok();
}

cbspmv_status_t cbspmv_export_csr(cbspmv_handle_t h, int64_t* row_ptr, int32_t* col_idx, double* val) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  const cb::Plan& p = h->plan;
  if (!row_ptr || (p.nnz && (!col_idx || !val))) return fail(CBSPMV_ERR_INVALID, "NULL output array");
  std::string msg;
  cbspmv_status_t st;
  if (p.lanes && h->device < 0) {
    st = cb::decode_lanes_to_csr(p.m, p.n, p.value_dtype, p.lane_units, p.lane_vals.data(), p.n_lane_vals,
                                 p.lane_words.data(), p.lane_words.size(), p.lane_gcols.data(), p.lane_gcols.size(),
                                 row_ptr, col_idx, val, p.nnz, &msg);
  } else if (p.lanes) {
    // read the device-resident lane stream back and decode it
    DeviceGuard g(h->device);
    CB_CUDA(g.err);
    std::vector<uint8_t> vals(h->lvals_count * (size_t)p.vsize);
    std::vector<uint64_t> words(h->lwords_count);
    std::vector<int32_t> gcols(h->lgcols_count);
    CB_CUDA(cudaDeviceSynchronize());
    if (!vals.empty()) CB_CUDA(cudaMemcpy(vals.data(), h->d_lvals, vals.size(), cudaMemcpyDeviceToHost));
    if (!words.empty()) CB_CUDA(cudaMemcpy(words.data(), h->d_lwords, words.size() * 8, cudaMemcpyDeviceToHost));
    if (!gcols.empty()) CB_CUDA(cudaMemcpy(gcols.data(), h->d_lgcols, gcols.size() * 4, cudaMemcpyDeviceToHost));
    st = cb::decode_lanes_to_csr(p.m, p.n, p.value_dtype, p.lane_units, vals.data(), h->lvals_count, words.data(),
                                 words.size(), gcols.data(), gcols.size(), row_ptr, col_idx, val, p.nnz, &msg);
  } else if (h->device < 0) {
    st = cb::decode_to_csr(p.m, p.n, p.value_dtype, p.aggregated, p.tiles, p.units, p.blob.data(), p.blob.size(),
                           p.stream.data(), p.stream.size(), p.restore_cols.data(), p.restore_cols.size(), row_ptr,
                           col_idx, val, p.nnz, &msg);
  } else {
    DeviceGuard g(h->device);
    CB_CUDA(g.err);
    std::vector<uint8_t> stream(h->stream_bytes);
    std::vector<CbTile> tiles(p.tiles.size());
    std::vector<int32_t> rcols(p.restore_cols.size());
    CB_CUDA(cudaDeviceSynchronize());
    if (!stream.empty()) CB_CUDA(cudaMemcpy(stream.data(), h->d_stream, stream.size(), cudaMemcpyDeviceToHost));
    if (!tiles.empty()) CB_CUDA(cudaMemcpy(tiles.data(), h->d_tiles, tiles.size() * sizeof(CbTile), cudaMemcpyDeviceToHost));
    if (!rcols.empty()) CB_CUDA(cudaMemcpy(rcols.data(), h->d_rcols, rcols.size() * 4, cudaMemcpyDeviceToHost));
    st = cb::decode_to_csr(p.m, p.n, p.value_dtype, p.aggregated, tiles, p.units, p.blob.data(), p.blob.size(),
                           stream.data(), stream.size(), rcols.data(), rcols.size(), row_ptr, col_idx, val, p.nnz,
                           &msg);
  }
  if (st != CBSPMV_OK) return fail(st, "%s", msg.c_str());
  return ok();
}

cbspmv_status_t cbspmv_export_blocked(cbspmv_handle_t h, int32_t* blk_row, int32_t* blk_col, int32_t* nnz_per_blk,
                                      uint8_t* type_per_blk, int64_t* cols_offset, int32_t* restore_cols) {
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  const cb::Plan& p = h->plan;
  for (size_t t = 0; t < p.tiles.size(); ++t) {
    if (blk_row) blk_row[t] = (int32_t)p.tiles[t].brow;
    if (blk_col) blk_col[t] = p.tile_bcol[t];
    if (nnz_per_blk) nnz_per_blk[t] = p.tiles[t].nnz;
    if (type_per_blk) type_per_blk[t] = p.tiles[t].fmt;
  }
  if (cols_offset && p.aggregated) std::memcpy(cols_offset, p.cols_offset.data(), p.cols_offset.size() * 8);
  if (restore_cols && p.aggregated) {
    if ((int64_t)p.restore_cols.size() >= p.restore_cols_len) {
      std::memcpy(restore_cols, p.restore_cols.data(), (size_t)p.restore_cols_len * 4);
    } else {   // built by the device analysis: resident on the device only
      DeviceGuard g(h->device);
      CB_CUDA(g.err);
      CB_CUDA(cudaDeviceSynchronize());
      CB_CUDA(cudaMemcpy(restore_cols, h->d_rcols, (size_t)p.restore_cols_len * 4, cudaMemcpyDeviceToHost));
    }
  }
  return ok();
}

// ---- CUDA-graph captured products -------------------------------------------------------
struct cbspmv_graph_s {
  uint32_t magic = 0xCB56A401u;
  int device = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

cbspmv_status_t cbspmv_graph_create(int count, const cbspmv_handle_t* hs, const int* k, const void* const* X,
                                    void* const* Y, const double* alpha, const double* beta, cbspmv_graph_t* out) {
  if (!out) return fail(CBSPMV_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (count < 1 || !hs) return fail(CBSPMV_ERR_INVALID, "count must be >= 1");
  for (int i = 0; i < count; ++i)
    if (!valid_handle(hs[i]) || hs[i]->device < 0) return fail(CBSPMV_ERR_INVALID, "problem %d: invalid or host-only handle", i);
  DeviceGuard g(hs[0]->device);
  CB_CUDA(g.err);
  CB_CUDA(cb::configure_kernels());
  // buffers the captured products will use are allocated before the capture
  for (int i = 0; i < count; ++i)
    if ((k ? k[i] : 1) >= 4 && !hs[i]->plan.lanes) {
      const cbspmv_status_t st = ensure_partial_multi(hs[i]);
      if (st != CBSPMV_OK) return st;
    }
  cudaStream_t s = nullptr;
  CB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  auto* G = new (std::nothrow) cbspmv_graph_s();
  if (!G) {
    cudaStreamDestroy(s);
    return fail(CBSPMV_ERR_OOM, "host allocation failed");
  }
  G->device = hs[0]->device;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  cbspmv_status_t st = CBSPMV_OK;
  std::string msg;
  if (e == cudaSuccess) {
    st = cbspmv_run_batched(count, hs, k, X, Y, alpha, beta, s);
    msg = g_err;
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    G->graph = graph;
    if (st == CBSPMV_OK && e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && st == CBSPMV_OK) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  cudaStreamDestroy(s);
  if (e != cudaSuccess || st != CBSPMV_OK) {
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
    if (st != CBSPMV_OK) return fail(st, "%s", msg.c_str());
    return fail(CBSPMV_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  *out = G;
  return ok();
}

cbspmv_status_t cbspmv_graph_launch(cbspmv_graph_t G, void* stream) {
  if (!G || G->magic != 0xCB56A401u) return fail(CBSPMV_ERR_INVALID, "invalid graph");
  DeviceGuard g(G->device);
  CB_CUDA(g.err);
  CB_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
  return ok();
}

cbspmv_status_t cbspmv_graph_destroy(cbspmv_graph_t G) {
  if (!G) return ok();
  if (G->magic != 0xCB56A401u) return fail(CBSPMV_ERR_INVALID, "invalid graph");
  DeviceGuard g(G->device);
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  G->magic = 0;
  delete G;
  return ok();
}

// ---- autotuned analysis --------------------------------------------------------------------
// Mean device time of one product on h (reps runs after two warm-up runs, one event pair).
static cbspmv_status_t time_handle(cbspmv_handle_t h, void* x, void* y, int reps, cudaStream_t s, double* ms) {
  for (int i = 0; i < 2; ++i) {
    cbspmv_status_t st = run_device(h, x, y, 1.0, 0.0, s);
    if (st != CBSPMV_OK) return st;
  }
  cudaEvent_t e0, e1;
  CB_CUDA(cudaEventCreate(&e0));
  CB_CUDA(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, s);
  for (int i = 0; i < reps && e == cudaSuccess; ++i)
    if (run_device(h, x, y, 1.0, 0.0, s) != CBSPMV_OK) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(CBSPMV_ERR_CUDA, "timing: %s", cudaGetErrorString(e));
  *ms = (double)t / reps;
  return ok();
}

cbspmv_status_t cbspmv_analyze_tuned(const cbspmv_csr_t* A, const cbspmv_opts_t* base, void* stream, int reps,
                                     cbspmv_handle_t* out, cbspmv_tune_report_t* rep) {
  if (!A || !out) return fail(CBSPMV_ERR_INVALID, "NULL argument");
  *out = nullptr;
  cbspmv_opts_t o0;
  if (base) o0 = *base; else cbspmv_default_opts(&o0);
  if (o0.device < 0) return fail(CBSPMV_ERR_INVALID, "tuning needs a device");
  if (reps < 1 || reps > 10000) return fail(CBSPMV_ERR_INVALID, "reps must be in [1, 10000]");
  cudaStream_t s = (cudaStream_t)stream;
  cbspmv_tune_report_t R{};
  // candidate options, tried one coordinate at a time from the paper's settings: column
  // aggregation (auto / off / on), unit size, then the format thresholds
  cbspmv_handle_t best = nullptr;
  cbspmv_opts_t best_o = o0;
  double best_ms = 0.0;
  void* x = nullptr;
  void* y = nullptr;
  auto consider = [&](const cbspmv_opts_t& o) -> cbspmv_status_t {
    cbspmv_handle_t h = nullptr;
    cbspmv_status_t st = cbspmv_analyze(A, &o, stream, &h);
    if (st != CBSPMV_OK) return st;
    DeviceGuard g(h->device);
    if (!x) {
      const size_t bytes = (size_t)(A->n > A->m ? A->n : A->m) * 8 + 16;
      if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess ||
          cudaMemsetAsync(x, 0, bytes, s) != cudaSuccess) {
        cbspmv_destroy(h);
        return fail(CBSPMV_ERR_OOM, "tuning buffers");
      }
    }
    double ms = 0.0;
    st = time_handle(h, x, y, reps, s, &ms);
    if (st != CBSPMV_OK) {
      cbspmv_destroy(h);
      return st;
    }
    if (R.n_tried < 16) {
      R.tried_ms[R.n_tried] = ms;
      R.tried_unit_work[R.n_tried] = o.unit_work;
      R.tried_col_agg[R.n_tried] = o.col_agg;
      R.tried_th1[R.n_tried] = o.th1;
      R.tried_th2[R.n_tried] = o.th2;
      R.tried_record_layout[R.n_tried] = o.record_layout;
    }
    R.n_tried++;
    if (!best || ms < best_ms) {
      if (best) cbspmv_destroy(best);
      best = h;
      best_ms = ms;
      best_o = o;
    } else {
      cbspmv_destroy(h);
    }
    return ok();
  };
  cbspmv_status_t st = consider(o0);
  if (st == CBSPMV_OK) {
    R.default_ms = best_ms;
    // the other side of the aggregation decision the default options took
    const int other = best->plan.aggregated ? 0 : 1;
    if (st == CBSPMV_OK && o0.col_agg != other) {
      cbspmv_opts_t o = best_o;
      o.col_agg = other;
      st = consider(o);
    }
    if (best->plan.lanes && st == CBSPMV_OK) {
      // lane-stream unit sizes (stored entries per unit)
      for (int uw : {1024, 4096})
        if (st == CBSPMV_OK) {
          cbspmv_opts_t o = best_o;
          o.unit_work = uw;
          st = consider(o);
        }
    }
    if (!o0.record_layout && !o0.plain_records && st == CBSPMV_OK) {
      // the record layout against the default lane-stream layout
      cbspmv_opts_t o = best_o;
      o.record_layout = 1;
      o.unit_work = 0;
      st = consider(o);
    }
    // the record layout's unit sizes and format thresholds (formats do not change the
    // lane-stream layout, which multiplies stored entries only)
    if (st == CBSPMV_OK && !best->plan.lanes) {
      for (int uw : {512, 768})
        if (st == CBSPMV_OK) {
          cbspmv_opts_t o = best_o;
          o.unit_work = uw;
          st = consider(o);
        }
      const int th[2][2] = {{16, 64}, {48, 192}};
      for (const auto& t : th)
        if (st == CBSPMV_OK) {
          cbspmv_opts_t o = best_o;
          o.th1 = t[0];
          o.th2 = t[1];
          st = consider(o);
        }
    }
  }
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (st != CBSPMV_OK) {
    std::string msg = g_err;
    if (best) cbspmv_destroy(best);
    return fail(st, "%s", msg.c_str());
  }
  R.best_ms = best_ms;
  R.best_unit_work = best_o.unit_work;
  R.best_col_agg = best_o.col_agg;
  R.best_th1 = best_o.th1;
  R.best_th2 = best_o.th2;
  R.best_record_layout = best_o.record_layout;
  if (rep) *rep = R;
  *out = best;
  return ok();
}

cbspmv_status_t cbspmv_get_stats(cbspmv_handle_t h, cbspmv_stats_t* s) {
  if (!valid_handle(h) || !s) return fail(CBSPMV_ERR_INVALID, "invalid handle or NULL stats");
  *s = h->plan.stats;
  return ok();
}

cbspmv_status_t cbspmv_destroy(cbspmv_handle_t h) {
  if (!h) return ok();
  if (!valid_handle(h)) return fail(CBSPMV_ERR_INVALID, "invalid handle");
  h->free_device();
  h->magic = 0;
  delete h;
  return ok();
}

const char* cbspmv_last_error(void) { return g_err.c_str(); }

// The run-kernel revision changes whenever the kernel's code changes (measurements taken
// with a profiler are tied to it).
const char* cbspmv_version(void) { return "cbspmv 0.6 (sm_103a; run kernel rev 21)"; }

}  // extern "C"

namespace cb {

bool server_run_args(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta, void* partial,
                     RunArgs* out, int* grid, int* n_slots, int* value_dtype) {
  if (!valid_handle(h)) return false;
  *out = run_args(h, x, y, alpha, beta);
  out->partial = partial;
  *grid = h->grid;
  *n_slots = h->plan.n_slots;
  *value_dtype = h->plan.value_dtype;
  return true;
}

bool noalloc_view(cbspmv_handle_t h, NoallocView* v) {
  if (!valid_handle(h)) return false;
  v->device = h->device;
  v->grid = h->grid;
  v->plan = &h->plan;
  RunArgs a{};
  a.stream = h->d_stream;
  a.tiles = h->d_tiles;
  a.rcols = h->d_rcols;
  a.units = h->d_units;
  a.blob = h->d_blob;
  a.worker_units = h->d_wunits;
  a.worker_off = h->d_woff;
  a.err = h->d_err;
  a.split_rows = h->d_split_rows;
  a.n_split_rows = (uint32_t)h->plan.split_rows.size();
  a.n_split_wide = (uint32_t)h->plan.n_split_wide;
  a.m = h->plan.m;
  a.n = h->plan.n;
  a.aggregated = h->plan.aggregated ? 1 : 0;
  a.value_dtype = h->plan.value_dtype;
  a.nvec = 1;
  a.ldx = h->plan.n;
  a.ldy = h->plan.m;
  a.lanes = h->plan.lanes ? 1 : 0;
  a.lunits = h->d_lunits;
  a.lvals = h->d_lvals;
  a.lwords = h->d_lwords;
  a.lgcols = h->d_lgcols;
  a.wait_budget = h->wait_budget;
  a.stuck_wait = h->stuck_wait;
  v->args = a;
  return true;
}

void set_last_error(const std::string& msg) { g_err = msg; }

cbspmv_status_t check_product_args(cbspmv_handle_t h, const void* x, const void* y) {
  const bool v = valid_handle(h);
  return check_run_args(h, 1, x, v ? h->plan.n : 0, y, v ? h->plan.m : 0);
}

}  // namespace cb
