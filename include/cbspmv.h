/*
 * cbspmv -- cache-friendly blocked sparse matrix-vector product for NVIDIA GB300 (sm_103a).
 *
 * The method is CB-SpMV (Cong, Sun, Chen, Xie, Liu, Qian, ICS '25): the matrix is cut
 * into independent 16x16 sub-blocks (Sec. 3.1); the coordinate bytes and values of each
 * sub-block are packed behind one virtual pointer (Sec. 3.2); sparse block rows get
 * block-aware column aggregation and every sub-block a COO / CSR / Dense format
 * (Sec. 3.3); the sub-blocks are spread over the GPU's workers by a priority-queue load
 * balance (Sec. 3.4, Algorithm 2); a kernel then forms y = alpha*A*x + beta*y
 * (Sec. 3.5, Algorithms 3 and 4).
 *
 * Conventions that hold for every call:
 *   - Every call returns a cbspmv_status_t. No call aborts, traps or prints; on failure
 *     cbspmv_last_error() holds a one-line message for the calling thread.
 *   - A handle owns all device memory it allocated until cbspmv_destroy(). Handles are
 *     not thread-safe: one host thread (or external locking) per handle.
 *   - Device pointers passed to run calls belong to the caller and must stay valid until
 *     the enqueued work has finished on the given stream. Run calls are asynchronous on
 *     that stream and do not synchronise the host (cbspmv_run_host is the exception).
 *   - cudaStream_t is passed as void* (NULL = the legacy default stream), so this header
 *     needs no CUDA include.
 *   - BLAS scaling: beta == 0 means y is not read (NaN/Inf in y are overwritten).
 *   - Matrices are canonical CSR: row_ptr non-decreasing from 0 to nnz, column indices
 *     strictly increasing inside each row and inside [0, n). Explicitly stored zeros are
 *     kept as entries. m, n < 2^31; nnz < 2^31.
 */
#ifndef CBSPMV_H_
#define CBSPMV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cbspmv_handle_s* cbspmv_handle_t;

typedef enum {
  CBSPMV_OK = 0,
  CBSPMV_ERR_INVALID = 1,        /* bad argument, size or handle */
  CBSPMV_ERR_NOT_CANONICAL = 2,  /* CSR not sorted / duplicate columns / index out of range */
  CBSPMV_ERR_OOM = 3,            /* host or device allocation failed */
  CBSPMV_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the CUDA error) */
  CBSPMV_ERR_TIMEOUT = 5,        /* a bounded device wait gave up (see cbspmv_check_device) */
  CBSPMV_ERR_UNSUPPORTED = 6,    /* option combination not implemented */
  CBSPMV_ERR_BUSY = 7            /* resource temporarily unavailable */
} cbspmv_status_t;

/* Storage type of the matrix values on the device. F64 is the reference path: values,
 * x, y and accumulation in IEEE double. F32, BF16 and F16 store the values in that type
 * (each FP64 input value rounded to nearest, ties to even, directly from FP64; overflow
 * gives an infinity) and use FP32 for x, y, alpha, beta and the accumulation: the
 * mixed-precision form the paper mentions (Sec. 2.2) without fixing its details. The
 * "vector type" of a handle is double for F64 and float for the other three. */
typedef enum { CBSPMV_F64 = 0, CBSPMV_F32 = 1, CBSPMV_BF16 = 2, CBSPMV_F16 = 3 } cbspmv_dtype_t;

/* Sub-block storage formats (Sec. 3.3.2). */
enum { CBSPMV_FMT_COO = 0, CBSPMV_FMT_CSR = 1, CBSPMV_FMT_DENSE = 2 };

/* A CSR matrix given by the caller. Values are always FP64 here; cbspmv_analyze copies
 * everything it needs, so the caller may free the arrays when the call returns.
 * on_device = 0: the three arrays are host pointers; on_device = 1: they are device
 * pointers. For the lane-stream layout on a device (record_layout 0 without
 * plain_records, or record_layout 2; device >= 0) with the arrays
 * in that device's memory, the analysis runs on that device from these arrays on the
 * given stream (GPU merge, tiling, aggregation and lane programs; units and load balance
 * on the host from the tile counts; Sec. 3.2-3.4, cost of Sec. 4.5). Otherwise the arrays
 * are copied to the host on the given stream and analysed there. */
typedef struct {
  int64_t m, n, nnz;
  const int64_t* row_ptr;   /* m + 1 entries */
  const int32_t* col_idx;   /* nnz entries */
  const double* val;        /* nnz entries */
  int on_device;
} cbspmv_csr_t;

/* Analysis options. Fill with cbspmv_default_opts() and override fields.
 *   th0: column aggregation is applied when the share of "super-sparse" 16x16
 *        sub-blocks (fewer than th1 nonzeros) exceeds th0 (Sec. 3.3.1; paper: 0.15).
 *   th1, th2: sub-block format thresholds, COO if nnz < th1, Dense if nnz > th2, CSR
 *        otherwise (Sec. 3.3.2; paper: 32 and 128). 0 <= th1 <= th2 <= 256.
 *   col_agg: -1 decide by th0, 0 never aggregate, 1 always aggregate.
 *   value_dtype: storage type of the values (CBSPMV_F64 for the FP64 path; see
 *        cbspmv_dtype_t for the reduced types).
 *   unit_work: target number of multiply-adds per scheduling unit (0 = default: 2,048
 *        stored entries in the lane-stream layout, or fewer, down to max(256, the largest
 *        block row), when the matrix has fewer such units than the handle has CTAs; 1,024
 *        multiply-adds in the record layout).
 *   load_balance: 1 (default) spread units over workers by the longest-first
 *        priority-queue rule; 0 deal them out round-robin in matrix order (ablation).
 *   device: CUDA device ordinal for the handle's memory; -1 builds a host-only handle
 *        (analysis, export and statistics work; run calls return CBSPMV_ERR_INVALID).
 *   keep_value_map: 0 (default) or 1, see cbspmv_update_values.
 *   record_layout: 0 (default): every value type is packed per unit in lane order (the
 *        lane-stream layout of the lane run kernel), except with plain_records = 1, which
 *        selects the record layout; 1: the per-sub-block record layout and its kernel;
 *        2: the lane-stream layout. Results agree within the tolerance of the value type. */
typedef struct {
  double th0;
  int th1, th2;
  int col_agg;
  cbspmv_dtype_t value_dtype;
  int unit_work;
  int load_balance;
  int device;
  int keep_value_map;       /* 1: record each entry's value slot (4 bytes per entry on the
                               device) so cbspmv_update_values can re-pack new values */
  int record_layout;        /* 0 default, 1 records, 2 lane streams (see above) */
  int plain_records;        /* 1: every sub-block record keeps the layout of Sec. 3.2 (no
                               values re-laid in load order): needed by cbspmv_spmm */
  int reserved[5];
} cbspmv_opts_t;

/* Statistics of an analysed matrix. Byte counts follow the storage model of Sec. 4.4.1
 * where noted. */
typedef struct {
  int64_t m, n, nnz;
  int64_t n_block_rows;
  int64_t n_tiles;                 /* non-empty 16x16 sub-blocks after aggregation */
  int64_t n_tiles_plain;           /* non-empty 16x16 sub-blocks without aggregation */
  double super_sparse_fraction;    /* share of plain sub-blocks with nnz < th1 */
  int aggregated;                  /* column aggregation applied (Sec. 3.3.1) */
  int value_dtype;
  int64_t n_fmt[3];                /* sub-blocks per format: COO, CSR, Dense */
  int64_t nnz_fmt[3];              /* stored entries per format */
  int64_t hist_coarse[8];          /* sub-block nnz histogram 1-32, 33-64, ..., 225-256 */
  int64_t hist_fine[4];            /* 1-8, 9-16, 17-24, 25-32 */
  int64_t restore_cols_len;        /* entries of restore_cols (without padding) */
  int64_t stream_bytes;            /* packed sub-block stream incl. alignment padding */
  int64_t metadata_bytes;          /* per-sub-block records as stored on the device */
  int64_t model_bytes_cb;          /* Sec. 4.4.1: nnzb*21 + nnz*9 (all-COO CB model) */
  int64_t model_bytes_csr;         /* Sec. 4.4.1: (m+1)*4 + nnz*12 */
  int64_t model_bytes_bsr16;       /* Sec. 4.4.1: 2048*nnzb + (blk_m+1)*4 + 4*nnzb */
  int64_t algo_bytes_per_run;      /* bytes model of one y = A x (beta = 0) */
  int64_t flops_per_run;           /* 2 * nnz */
  int64_t mults_per_run;           /* multiply-adds issued incl. Dense zero fill */
  int64_t n_units, n_split_units, n_split_rows, n_workers;
  double worker_load_max, worker_load_mean, worker_load_std;  /* multiply-adds per worker */
  double tb8_load_std;             /* per-thread-block (8 sub-blocks) nnz std, Algorithm 2 order */
  double analyze_ms;               /* wall time of the analysis (host, or GPU kernels and host steps) */
  int64_t n_entry_mode_units;      /* units scheduled in single entries (sparse pieces) */
  int64_t n_xseq_units;            /* units whose chunks all cover consecutive columns */
  int64_t fma_slots;               /* FMA slots the run kernel's walks issue per vector (32 lanes x
                                      chunk steps x chunk size, summed over units); nnz / fma_slots
                                      is the fraction of FMA issue that does useful work */
  int64_t n_direct_units;          /* units whose chunk descriptors hold value offsets and columns */
  int64_t lane_layout;             /* 1: lane-stream layout (see record_layout), 0: records */
  int64_t analyzed_on_device;      /* 1: built on the GPU from a device CSR (cbspmv_csr_t) */
  int64_t n_g16_units;             /* lane-stream units whose gather lists are uint16 offsets */
  int64_t gather_list_bytes;       /* lane-stream gather-list bytes one product reads */
} cbspmv_stats_t;

/* Fills *opts with the paper's settings: th0 0.15 (Sec. 3.3.1), th1 32 and th2 128
 * (Sec. 3.3.2), col_agg -1 (the paper's rule), FP64 values (its evaluation, Sec. 4.1),
 * default unit size, load balance on (Sec. 3.4), device 0. Errors: CBSPMV_ERR_INVALID
 * (NULL). */
cbspmv_status_t cbspmv_default_opts(cbspmv_opts_t* opts);

/* Analyses a CSR matrix (Sec. 3 overview; Sec. 3.1-3.4): validation, 16x16 tiling, the
 * column-aggregation decision and aggregation, per-sub-block format selection, packing
 * into one byte stream with 16-byte aligned virtual pointers, units of work and their
 * load-balanced assignment to the kernel's workers; then one upload per device array.
 * stream: upload stream (void* cudaStream_t); the call synchronises it before returning.
 * The host analysis runs on all hardware threads (at most 64), or on the number given by
 * the environment variable CBSPMV_HOST_THREADS (1..64); its result does not depend on it.
 * On success *out is a new handle. Errors: CBSPMV_ERR_INVALID (NULL pointers, sizes),
 * CBSPMV_ERR_NOT_CANONICAL, CBSPMV_ERR_OOM, CBSPMV_ERR_CUDA, CBSPMV_ERR_UNSUPPORTED. A failed
 * call frees everything it allocated. Fault injection for tests: when the environment
 * variable CBSPMV_FAIL_ALLOC_AFTER holds N >= 0, the call's device allocation number N
 * (from 0) fails as out of memory. */
cbspmv_status_t cbspmv_analyze(const cbspmv_csr_t* A, const cbspmv_opts_t* opts, void* stream,
                               cbspmv_handle_t* out);

/* y = alpha * A * x + beta * y on the device (Sec. 3.5, Algorithms 3 and 4).
 * x: device array of n values, y: device array of m values, both of the handle's
 * vector type (double for CBSPMV_F64, float for F32, BF16 and F16), aligned to the
 * element size; y must not overlap x. Enqueued on `stream`, no host synchronisation. One kernel
 * launch, plus a second small one that adds the parts of block rows the analysis cut into
 * several units (when there are any). Concurrent runs on one handle must be serialised on
 * one stream (they share the handle's partial-sum buffer). Errors: CBSPMV_ERR_INVALID, CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_run(cbspmv_handle_t h, const void* x, void* y, double alpha, double beta,
                           void* stream);

/* The product of Sec. 3.5 end to end from host memory (the paper times the kernel alone;
 * this is the call a host-side user makes): copies x (n values of the handle's
 * vector type) to the device, runs, copies y back (m values; read first when beta != 0),
 * then synchronises the stream. x_host / y_host may be pageable or pinned. Uses staging
 * buffers owned by the handle (allocated on first use). */
cbspmv_status_t cbspmv_run_host(cbspmv_handle_t h, const void* x_host, void* y_host,
                                double alpha, double beta, void* stream);

/* Y = alpha * A * X + beta * Y for k right-hand sides (the multiple-vector form of the
 * product of Sec. 2.2; the paper evaluates one vector). X: device array, column-major
 * n x k with leading dimension ldx >= n (column j at X + j * ldx); Y: device array,
 * column-major m x k with ldy >= m. Element type, alignment and the no-overlap rule
 * (between the whole spans of X and Y) are those of cbspmv_run; k = 0 does nothing.
 * Reduced value types: the columns are computed in passes of 4 (then 2, then 1) vectors
 * in the record layout, of 4 (then 1) in the lane-stream layout, except for matrices of 2^22
 * or more stored entries whose gathered x slots serve fewer than two entries each
 * (16 x sub-blocks > nnz / 2: one column per pass, since a pass gathers every slot once
 * per vector): each pass reads every
 * unit of the matrix once and multiplies it into all its vectors, so the matrix is read
 * ceil(k/4)-ish times instead of k times. FP64 values in the lane-stream
 * layout: one column per pass, since the FP64 FMA pipe, not the matrix bytes, bounds the
 * product (a pass over several vectors measured slower per vector). Each column is computed exactly as
 * cbspmv_run would (same summation order, so the results are bitwise equal to k separate
 * runs). The first call with k > 1 allocates a partial-sum buffer for 4-vector passes,
 * owned by the handle. Errors: CBSPMV_ERR_INVALID (k < 0, ldx < n, ldy < m, NULL or
 * misaligned arrays, overlap), CBSPMV_ERR_OOM, CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_run_multi(cbspmv_handle_t h, int k, const void* X, int64_t ldx, void* Y,
                                 int64_t ldy, double alpha, double beta, void* stream);

/* Y = alpha * A * X + beta * Y for k right-hand sides on the tensor cores (the multi-vector
 * form of the product of Sec. 3.5; with k vectors each 16x16 sub-block of Sec. 3.1 becomes
 * a contraction of shape 16 x 16 x k). X: device array, row-major n x k with leading
 * dimension ldx >= k (element (i, j) at X[i * ldx + j]); Y: row-major m x k, ldy >= k; FP32
 * (the vector type of BF16 handles), 4-byte aligned, not overlapping. Requires a device
 * handle with BF16 values in the record layout analysed with opts.plain_records = 1
 * (CBSPMV_ERR_UNSUPPORTED otherwise; other value types and layouts use cbspmv_run_multi). Each sub-block is expanded to a
 * zero-filled 16x16 BF16 tile and multiplied with mma.sync.m16n8k16 (BF16 inputs, FP32
 * accumulation); every x is split exactly into three BF16 parts (|x - sum| <= 2^-25 |x|) so
 * the products keep FP32 accuracy; a row's result has error at most gamma_{6r + 16} with
 * u = 2^-23 times sum_j |a_ij x_j| (r = stored entries of the row). Per 32 columns one
 * pass splits X into a workspace (8 bytes per x) and one launch multiplies (the matrix is
 * read once per 32 columns), plus one small launch that adds the segments of block rows
 * with more than 64 sub-blocks. The first call builds the segment list and allocates a
 * partial-sum buffer, and the split-X workspace grows to n x 32 x 8 bytes at most (both
 * owned by the handle and shared by its calls: calls on one handle whose work may overlap on
 * the GPU, on other streams, race, so serialise them). Like
 * Dense zero fill, a non-finite x reaches every row of a sub-block holding its column.
 * Asynchronous on `stream`. Errors: CBSPMV_ERR_INVALID (arguments), CBSPMV_ERR_UNSUPPORTED,
 * CBSPMV_ERR_OOM, CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_spmm(cbspmv_handle_t h, int k, const void* X, int64_t ldx, void* Y,
                            int64_t ldy, double alpha, double beta, void* stream);

/* Batched analysis (the paper analyses one matrix; this is the many-matrix form of
 * cbspmv_analyze, Sec. 3): count matrices with the same options (cbspmv_analyze on each of
 * A[0..count)).
 * out: array of count handles, all set to NULL first. On failure every handle created by
 * the call is destroyed, out[] stays NULL and the message names the failing matrix.
 * count = 0 does nothing. Errors: those of cbspmv_analyze, CBSPMV_ERR_INVALID for
 * count < 0 or NULL arrays. */
cbspmv_status_t cbspmv_analyze_batched(int count, const cbspmv_csr_t* A,
                                       const cbspmv_opts_t* opts, void* stream,
                                       cbspmv_handle_t* out);

/* Batched product (the paper runs one product per launch; this is the many-matrix form of
 * the product of Sec. 3.5): count independent products on one stream; for problem i,
 * Y[i] = alpha[i] * A_i * X[i] + beta[i] * Y[i] with k[i] right-hand sides stored
 * column-major and packed (leading dimensions n_i and m_i); k may be NULL (one vector
 * each). Every problem's arguments are checked before any work is enqueued; a failing
 * check enqueues nothing and the message names the problem. All handles must belong to
 * one device. The products of all problems run in one persistent launch of the run
 * kernel per value type and per 64 products (each CTA works through its share of every
 * problem, as given by each problem's load balance), plus one small launch that adds the
 * parts of split block rows; a handle that appears more than once, or with k > 1, has its
 * further products in further launches (they share its partial-sum buffer). Handles other
 * than FP64 lane streams take their columns in passes of four where they can (one launch
 * multiplies each unit into four columns), the rest one at a time; the
 * first such call allocates the handle's 4-vector partial-sum buffer. Every
 * product is computed exactly as cbspmv_run computes it, so results are bitwise equal to
 * separate runs. Errors: as cbspmv_run_multi. */
cbspmv_status_t cbspmv_run_batched(int count, const cbspmv_handle_t* h, const int* k,
                                   const void* const* X, void* const* Y, const double* alpha,
                                   const double* beta, void* stream);

/* The product of cbspmv_run with no allocation of any kind. The paper has no counterpart:
 * this entry point exists for callers that may not call cudaMalloc, cudaFree or any
 * allocating routine when they run the product, for example code whose device memory
 * is owned by another allocator (a framework's memory pool) or code on a latency-critical
 * path where an allocation, which can synchronise the device, is not acceptable.
 * Arguments, layouts and the result are those of cbspmv_run; h must be a device handle.
 * Scratch: the partial sums of block rows cut into several units come from one fixed array
 * in the library's device image (7.75 MiB, held by every GPU that loads the library until
 * the process exits): at most 63,488 partial-sum slots (cbspmv_get_stats: n_split_units);
 * larger matrices are rejected with CBSPMV_ERR_INVALID. The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture. Every call writes each slot it reads before reading it, so no
 * clearing is needed, but all calls share the array: calls whose work overlaps on the GPU
 * (other streams, other handles, other host threads) race and give wrong results, so
 * serialise them. Device-side wait errors go to
 * the handle's error word (cbspmv_check_device). */
cbspmv_status_t cbspmv_run_noalloc(cbspmv_handle_t h, const void* x, void* y, double alpha,
                                   double beta, void* stream);

/* ---- CUDA graphs (the paper has no counterpart) -------------------------------------------
 * Captures the launches of cbspmv_run_batched with these arguments (same meaning and
 * checks) into an instantiated CUDA graph; cbspmv_graph_launch replays them on a stream
 * with one graph launch. The graph keeps the handles' device arrays and the X / Y
 * pointers: replays read the current contents of X and overwrite Y. The handles must
 * outlive the graph. Errors: those of cbspmv_run_batched, CBSPMV_ERR_CUDA. */
typedef struct cbspmv_graph_s* cbspmv_graph_t;
/* Capture (no counterpart in the paper). */
cbspmv_status_t cbspmv_graph_create(int count, const cbspmv_handle_t* h, const int* k,
                                    const void* const* X, void* const* Y, const double* alpha,
                                    const double* beta, cbspmv_graph_t* out);
/* Replays the captured products on `stream` (no counterpart in the paper). Errors:
 * CBSPMV_ERR_INVALID (invalid graph), CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_graph_launch(cbspmv_graph_t g, void* stream);
/* Frees the graph (no counterpart in the paper); NULL is accepted. */
cbspmv_status_t cbspmv_graph_destroy(cbspmv_graph_t g);

/* ---- Autotuned analysis ------------------------------------------------------------------
 * The thresholds of Sec. 3.3 are heuristics (th0 0.15, th1 32, th2 128). This call analyses
 * A with the given options, then varies one choice at a time, keeping the fastest so far:
 * column aggregation (auto / off / on: th0 only ever decides between these two layouts, so
 * they stand for every th0); for a lane-stream layout the unit size (1024, 4096 stored
 * entries); the record layout (record_layout = 1) against the default lane streams; for
 * the record layout the unit size (512, 768 multiply-adds) and the format thresholds
 * (th1, th2) = (16, 64) and (48, 192). The 16x16 sub-block is fixed (the 4-bit coordinates
 * of Sec. 3.2) and so is the number of warps per CTA (set per kernel and value type). Each
 * candidate is timed over `reps` products (1..10000) on the device. *out is the fastest
 * handle; *rep (may be NULL) lists the candidates. base->device must be a device. Every
 * handle computes the same product (only the layout differs). Errors: those of
 * cbspmv_analyze, CBSPMV_ERR_CUDA. */
typedef struct {
  int n_tried;
  double default_ms, best_ms;
  int best_unit_work, best_col_agg, best_th1, best_th2;
  double tried_ms[16];
  int tried_unit_work[16], tried_col_agg[16], tried_th1[16], tried_th2[16];
  int best_record_layout;
  int tried_record_layout[16];
} cbspmv_tune_report_t;
/* Tuned analysis: the heuristics of Sec. 3.3 searched by timing (the paper fixes them). */
cbspmv_status_t cbspmv_analyze_tuned(const cbspmv_csr_t* A, const cbspmv_opts_t* base,
                                     void* stream, int reps, cbspmv_handle_t* out,
                                     cbspmv_tune_report_t* report);

/* Replaces the values of an analysed matrix whose sparsity pattern is unchanged (the case
 * that amortises the analysis of Sec. 3 over repeated products, Sec. 4.5): val holds the
 * new FP64 values in the order of the CSR given to cbspmv_analyze (nnz entries; host
 * pointer when on_device = 0, device pointer when 1). The values are converted to the
 * handle's storage type exactly as the analysis converts them and written into the packed
 * records on the device by one kernel; the blocked structure is unchanged, so every later
 * product and export is that of a fresh analysis of the new values. Requires a device
 * handle analysed with opts.keep_value_map = 1. Asynchronous on `stream` (a host array
 * is copied through a staging buffer owned by the handle, allocated on first use).
 * Errors: CBSPMV_ERR_INVALID (NULL val with nnz > 0, no value map), CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_update_values(cbspmv_handle_t h, const double* val, int on_device,
                                     void* stream);

/* Measurement support (the paper has no counterpart): runs the product of cbspmv_run
 * `reps` times (1..100000) on `stream`, with CUDA events recorded on that stream around
 * each of its kernel launches, and returns the mean device time per run of the main run
 * kernel (*ms_main) and of the kernel that adds the parts of split block rows
 * (*ms_combine, 0 when there are none), plus the number of kernel launches one run makes
 * (*launches_per_run: 0, 1 or 2). Synchronises `stream`. Arguments and results otherwise
 * as cbspmv_run. Errors: as cbspmv_run, CBSPMV_ERR_INVALID for reps out of range. */
cbspmv_status_t cbspmv_time_kernels(cbspmv_handle_t h, const void* x, void* y, double alpha,
                                    double beta, int reps, void* stream, double* ms_main,
                                    double* ms_combine, int* launches_per_run);

/* Measurement support (the paper has no counterpart): the FP64 FMA rate of `device`, the
 * roofline of the FP64 run kernel, which issues one FP64 FMA per stored entry. Runs a
 * kernel of independent FMA chains (one CTA per SM) on `stream`, synchronises it, and
 * returns the achieved rate (*gflops, 2 flops per FMA, at the clock the device runs at)
 * and the SM cycles one warp-wide FP64 FMA occupies its SM sub-partition
 * (*cycles_per_warp_fma). Allocates and frees a few KB of device memory.
 * Errors: CBSPMV_ERR_INVALID (NULL outputs), CBSPMV_ERR_OOM, CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_measure_fp64_fma(int device, void* stream, double* gflops,
                                        double* cycles_per_warp_fma);

/* ---- Serving (the paper has no serving system; it motivates its preprocessing cost by
 * repeated products as in iterative solvers, Sec. 4.5) ---------------------------------
 * A server keeps analysed matrices resident on one device and runs requests submitted
 * from any host thread: y = alpha*A*x + beta*y products and CG solves of A x = b for
 * symmetric positive definite A. A background engine thread admits queued requests in
 * arrival order while a slot (max_inflight) and device memory (memory_budget, a pool the
 * server allocates once) are free (a CG request beyond max_inflight_cg solves in flight
 * keeps its place while later products are admitted), and advances every in-flight request by one step per
 * tick: the products of all in-flight requests run as one batched launch of the run kernel
 * per value type (see cbspmv_run_batched), the CG vector steps as batched kernels; a solve
 * in its inner CG phase runs up to inner_steps inner iterations per tick (its scalars stay
 * on the device, and the steps after its inner convergence do nothing; with
 * cg_oldest_first the older solves run more of them, which brings the serving of long
 * solves closer to arrival order). Each result is the same whether the request runs alone
 * or among others, and with either option.
 * CG (mixed precision with FP64 refinement): r = b - A x and x += d in FP64 with the
 * FP64-value product; each correction A d = r is solved by CG on cg_inner_dtype values
 * (FP32 vectors and accumulation for the reduced types; FP64 for CBSPMV_F64) until its
 * residual is max(inner_tol, 0.3 tol ||b|| / ||r||) times its start, r being the FP64
 * residual the correction starts from (the first correction, r = b, stops at
 * max(inner_tol, 0.3 tol), a later one as soon as it closes the gap to tol); the solve ends when
 * ||b - A x|| <= tol ||b|| (FP64). */
typedef struct cbspmv_server_s* cbspmv_server_t;

typedef struct {
  int device;               /* CUDA device of the server and its matrices */
  int64_t memory_budget;    /* bytes of request workspace (allocated at creation) */
  int max_inflight;         /* requests in flight, 1..64 (1 = one request at a time) */
  cbspmv_dtype_t cg_inner_dtype;  /* values of the inner CG product (default BF16) */
  double inner_tol;         /* inner CG: stop at ||r|| <= inner_tol ||r0|| at the tightest
                               (default 1e-4; see above for later corrections) */
  int inner_max_iter;       /* inner CG iterations per correction (default 2000) */
  int max_outer;            /* refinement steps before a solve fails (default 30) */
  int inner_steps;          /* inner CG iterations per engine tick, 1..64 (default 8; 0 = 8) */
  int max_inflight_cg;      /* CG solves in flight at most (0 = max_inflight); products keep
                               being admitted past CG requests that wait for this limit */
  int cg_oldest_first;      /* 1: per tick the oldest solve in its inner phase runs all
                               inner_steps iterations, the next inner_steps / 2, the others
                               inner_steps / 4 (at least 1); 0 (default): all inner_steps */
  int reserved[5];
} cbspmv_server_opts_t;

enum { CBSPMV_REQ_SPMV = 0, CBSPMV_REQ_CG = 1 };

/* A request. SPMV: in = x (n doubles, host), out = y (m doubles, host; read first when
 * beta != 0). CG: in = b (n doubles), out = x (n doubles), tol = relative residual
 * target (e.g. 1e-8). Host buffers must stay valid until the request is done. */
typedef struct {
  int kind;
  int matrix;               /* id from cbspmv_server_register */
  const double* in;
  double* out;
  double alpha, beta;       /* SPMV only */
  double tol;               /* CG only */
  int reserved[4];
} cbspmv_request_t;

typedef struct {
  int done;                 /* 1 when finished (out written) */
  cbspmv_status_t status;   /* CBSPMV_OK, CBSPMV_ERR_TIMEOUT (CG did not converge within
                               max_outer refinements) or CBSPMV_ERR_CUDA */
  int iterations;           /* CG: inner iterations in total */
  int refinements;          /* CG: FP64 refinement steps after the first residual */
  double rel_residual;      /* CG: ||b - A x|| / ||b|| measured in FP64 at the end */
  double t_submit, t_admit, t_done;   /* host steady-clock seconds */
} cbspmv_result_t;

typedef struct {
  int64_t submitted, admitted, completed, ticks, launches;
  int64_t max_inflight_seen, arena_used_max, arena_capacity, queued, inflight;
} cbspmv_server_stats_t;

/* Server defaults (no counterpart in the paper): device 0, 4 GiB budget, 64 in flight,
 * BF16 inner values, inner_tol 1e-4, 2000 inner iterations, 30 refinements, 8 inner
 * iterations per tick, no separate limit on CG solves in flight. */
cbspmv_status_t cbspmv_server_default_opts(cbspmv_server_opts_t* opts);
/* Creates a server (no counterpart in the paper; the repeated products that amortise the
 * analysis, Sec. 4.5): allocates the memory budget, a stream and the engine thread.
 * Errors: CBSPMV_ERR_INVALID (options), CBSPMV_ERR_OOM, CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_server_create(const cbspmv_server_opts_t* opts, cbspmv_server_t* out);
/* Registers a matrix with the server (the analysis of Sec. 3, kept resident): analyses A
 * (opts as cbspmv_analyze; device and value type are the server's) with FP64
 * values and, for a square A, also with cg_inner_dtype values (in the lane-stream layout
 * unless opts.record_layout asks otherwise); the matrices stay resident until
 * cbspmv_server_destroy. *matrix_id names it in requests (at most 1024). */
cbspmv_status_t cbspmv_server_register(cbspmv_server_t s, const cbspmv_csr_t* A,
                                       const cbspmv_opts_t* opts, int* matrix_id);
/* Queues a request (no counterpart in the paper); *ticket identifies it. Errors: CBSPMV_ERR_INVALID (unknown matrix,
 * NULL buffers, CG on a non-square matrix, tol <= 0), CBSPMV_ERR_OOM (the request's device
 * workspace is larger than the whole memory budget, so it could never be admitted; nothing
 * is queued), CBSPMV_ERR_CUDA (engine stopped). */
cbspmv_status_t cbspmv_server_submit(cbspmv_server_t s, const cbspmv_request_t* req,
                                     uint64_t* ticket);
/* Polls a request (no counterpart in the paper). Non-blocking: *res = the request's state (res->done = 0 while it runs). A finished
 * request's ticket is released by the call that reports it done. */
cbspmv_status_t cbspmv_server_poll(cbspmv_server_t s, uint64_t ticket, cbspmv_result_t* res);
/* Waits for a request (no counterpart in the paper): up to timeout_ms; CBSPMV_ERR_TIMEOUT if it is still running (the
 * ticket stays valid). */
cbspmv_status_t cbspmv_server_wait(cbspmv_server_t s, uint64_t ticket, int timeout_ms,
                                   cbspmv_result_t* res);
/* Counters of the server (no counterpart in the paper): requests submitted, admitted and
 * completed, engine ticks and launches, the most requests in flight and the arena use.
 * Errors: CBSPMV_ERR_INVALID (invalid server or NULL stats). */
cbspmv_status_t cbspmv_server_get_stats(cbspmv_server_t s, cbspmv_server_stats_t* stats);
/* Stops the engine (requests still queued or in flight are abandoned), frees everything
 * (no counterpart in the paper). NULL is accepted. */
cbspmv_status_t cbspmv_server_destroy(cbspmv_server_t s);

/* Failure detection (no counterpart in the paper): reads the handle's device error word
 * (set by bounded device-side waits that gave up)
 * and clears it: CBSPMV_OK or CBSPMV_ERR_TIMEOUT. Synchronises `stream`. The record-layout
 * kernel waits for its own bulk copies with a budget of 4e9 SM cycles (about 2 s), or the
 * number in the environment variable CBSPMV_WAIT_BUDGET_CYCLES when the handle was analysed;
 * a warp whose wait gave up records the error, waits for its copies with the full budget
 * and stops, so the product is incomplete but the device stays usable. Test hook: with
 * CBSPMV_TEST_STUCK_WAIT=1 at analysis, each warp's first wait of the record kernel is on
 * a barrier nothing arrives at, so it runs out of its budget. The lane-stream kernel has no
 * such wait. */
cbspmv_status_t cbspmv_check_device(cbspmv_handle_t h, void* stream);

/* Reconstructs the CSR matrix from the handle's device-resident blocked format: the
 * inverse of the packing of Sec. 3.2-3.3, which loses no entry (bit-exact round trip of
 * row_ptr, col_idx and the value bits for FP64 values; for the reduced types, the stored
 * values widened exactly to double). Host output arrays of m+1, nnz, nnz entries; the
 * caller owns them. Synchronous (reads the device arrays back). Errors:
 * CBSPMV_ERR_INVALID (invalid handle, NULL arrays, an inconsistent layout),
 * CBSPMV_ERR_CUDA. */
cbspmv_status_t cbspmv_export_csr(cbspmv_handle_t h, int64_t* row_ptr, int32_t* col_idx,
                                  double* val);

/* The high-level metadata of Sec. 3.1 in matrix (row-major) order, before the load
 * balance: per sub-block its block row, block column (the aggregated block column when
 * aggregation is on), nnz and format; and the aggregation arrays of Sec. 3.3.1
 * (cols_offset: n_block_rows + 1 entries; restore_cols: stats.restore_cols_len entries).
 * Any output pointer may be NULL. Host arrays sized from cbspmv_get_stats(). */
cbspmv_status_t cbspmv_export_blocked(cbspmv_handle_t h, int32_t* blk_row, int32_t* blk_col,
                                      int32_t* nnz_per_blk, uint8_t* type_per_blk,
                                      int64_t* cols_offset, int32_t* restore_cols);

/* Statistics of the analysis into *stats (host struct, caller-owned): the storage model
 * of Sec. 4.4.1 (CB, CSR and 16x16 BSR bytes), the sub-block nnz histogram of Fig. 3, the
 * per-thread-block load spread of Fig. 4 and Algorithm 2, the format mix of Sec. 3.3.2,
 * the column-aggregation decision of Sec. 3.3.1, the host analysis time of Sec. 4.5, and
 * this library's units, workers, bytes model and FMA slot count. No device access.
 * Errors: CBSPMV_ERR_INVALID (invalid handle or NULL stats). */
cbspmv_status_t cbspmv_get_stats(cbspmv_handle_t h, cbspmv_stats_t* stats);

/* Frees the handle and all its device memory (synchronises the device first); the paper
 * has no counterpart (handle lifetime of this library). NULL is accepted.
 * Errors: CBSPMV_ERR_INVALID (a pointer that is not a live handle). */
cbspmv_status_t cbspmv_destroy(cbspmv_handle_t h);

/* Message of the last failed call on this host thread ("" if none); the paper has no
 * counterpart (error reporting of this library). The string is owned by the library and
 * valid until the thread's next call. */
const char* cbspmv_last_error(void);

/* Library version string, including the run kernel's revision ("run kernel rev N"); the
 * paper has no counterpart. Owned by the library. */
const char* cbspmv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CBSPMV_H_ */
