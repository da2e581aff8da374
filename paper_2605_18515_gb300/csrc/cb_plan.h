// Host-side result of the analysis (Sec. 3): everything that is uploaded to the device,
// plus host copies kept for export and statistics. C++ only, no CUDA types.
#ifndef CB_PLAN_H_
#define CB_PLAN_H_
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <functional>
#include <vector>

#include "../../include/cbspmv.h"
#include "cb_layout.h"

namespace cb {
// The lane-stream layout unless the options ask for the record layout (record_layout 1, or
// the default with plain_records, which only the record layout has).
inline bool uses_lanes(const cbspmv_opts_t& o) {
  return o.record_layout == 2 || (o.record_layout == 0 && !o.plain_records);
}
}  // namespace cb

namespace cb {

// Allocator whose value-initialisation of new elements is a no-op: for buffers that are
// written in full before they are read (the packed stream is 0.8 GB for the FEM workload;
// zero-filling it on one thread cost more than a third of the packing).
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U, class... Args>
  void construct(U* p, Args&&... args) { ::new ((void*)p) U(std::forward<Args>(args)...); }
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) { ::new ((void*)p) U; }
};
using ByteBuf = std::vector<uint8_t, NoInitAlloc<uint8_t>>;

struct Plan {
  int64_t m = 0, n = 0, nnz = 0;
  int64_t nbr = 0;                 // block rows
  int value_dtype = CBSPMV_F64;
  int vsize = 8;                   // bytes per stored value
  bool aggregated = false;
  double th0 = 0.15;
  int th1 = 32, th2 = 128;

  std::vector<CbTile> tiles;       // row-major order (block row, then block column)
  std::vector<int32_t> tile_bcol;  // block column per tile (aggregated index when aggregated)
  ByteBuf stream;                  // packed records (size multiple of 16; every byte written)
  std::vector<int32_t> restore_cols;  // with CB_RC_PAD zero entries appended
  std::vector<int64_t> cols_offset;   // nbr + 1 (aggregated only)
  int64_t restore_cols_len = 0;

  std::vector<CbUnit> units;
  std::vector<uint32_t, NoInitAlloc<uint32_t>> sched;   // lane schedules of all units (see cb_layout.h;
                                                      // each unit zeroes its own range)
  ByteBuf blob;                        // unit blobs (see cb_layout.h; every byte written)
  std::vector<CbSplitRow> split_rows;  // block rows cut into several units
  std::vector<uint32_t> worker_units;  // unit ids grouped by worker (CTA)
  std::vector<uint32_t> worker_off;    // n_workers + 1
  std::vector<uint32_t> value_slot;    // per CSR entry: stream offset of its value / vsize (optional)
  int n_workers = 0;
  int n_split_rows = 0;
  int n_split_wide = 0;                // the last split rows, with > CB_COMBINE_WIDE_PARTS parts
  int64_t fma_slots = 0;               // FMA slots the walks of all units issue (one vector)
  int n_slots = 0;

  // Lane-stream layout (FP64 values; see cb_layout.h): replaces the record stream, the lane
  // schedules and the unit blobs on the device. lane_units are in worker order like units;
  // the three arrays are host copies, released once uploaded to a device.
  bool lanes = false;
  std::vector<CbLaneUnit> lane_units;
  ByteBuf lane_vals;                    // values in the storage type (n_lane_vals of them)
  std::vector<uint64_t, NoInitAlloc<uint64_t>> lane_words;
  std::vector<int32_t, NoInitAlloc<int32_t>> lane_gcols;
  size_t n_lane_vals = 0, n_lane_words = 0, n_lane_gcols = 0;   // element counts of the three arrays

  cbspmv_stats_t stats{};
};

// Validates the CSR and fills *plan. n_workers: number of persistent CTAs the kernel will
// launch (the load balance assigns units to them). Returns CBSPMV_OK or an error with
// *msg set.
cbspmv_status_t analyze_host(const cbspmv_csr_t& A, const cbspmv_opts_t& opts, int n_workers,
                             Plan* plan, std::string* msg);

// Steps of the analysis shared by the host analysis and the device analysis of
// analyze_dev.cu (which builds p.tiles, the block-row tile offsets and the aggregation on
// the GPU, and the lane programs there too).
void cut_units(Plan& p, const std::vector<int64_t>& tile_off, const cbspmv_opts_t& opts, int n_workers);
cbspmv_status_t check_units(const Plan& p, std::string* msg);
void balance_units(Plan& p, const cbspmv_opts_t& opts, int n_workers, std::vector<double>* load);
cbspmv_status_t lane_offsets(Plan& p, std::vector<uint64_t>* voff, std::vector<uint64_t>* woff,
                             std::vector<uint64_t>* goff, std::string* msg);
void fill_stats(Plan& p, int64_t plain_tiles, double frac, const std::vector<double>& load);
cbspmv_status_t validate_shape(const cbspmv_csr_t& A, std::string* msg);
// f(lo, hi) over [0, n) in chunks of grain on all host cores
void host_parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& f);
// sub-block format of a tile with nnz entries (Sec. 3.3.2): COO below th1, Dense above th2
int tile_format(int nnz, int th1, int th2);
cbspmv_status_t check_opts(const cbspmv_opts_t& opts, int n_workers, std::string* msg);

// Rebuilds CSR from the packed layout (host arrays). Used by export on both host-only
// handles and on data read back from the device. Stored values are widened exactly to FP64.
// units and blob (the unit blobs with their lane schedules) locate the values of direct
// units, which are stored in load order after the coordinate parts.
cbspmv_status_t decode_to_csr(int64_t m, int64_t n, int value_dtype, bool aggregated,
                              const std::vector<CbTile>& tiles, const std::vector<CbUnit>& units,
                              const uint8_t* blob, size_t blob_size, const uint8_t* stream,
                              size_t stream_size, const int32_t* restore_cols,
                              size_t restore_len, int64_t* row_ptr, int32_t* col, double* val,
                              int64_t nnz_expected, std::string* msg);

// Rebuilds CSR from the lane-stream layout (host arrays: the units in worker order and
// their values (nvals of the storage type), entry words and gather lists, as described in
// cb_layout.h). Stored values are widened exactly to FP64.
cbspmv_status_t decode_lanes_to_csr(int64_t m, int64_t n, int value_dtype, const std::vector<CbLaneUnit>& units,
                                    const uint8_t* vals, size_t nvals, const uint64_t* words, size_t nwords,
                                    const int32_t* gcols, size_t ngcols, int64_t* row_ptr, int32_t* col,
                                    double* val, int64_t nnz_expected, std::string* msg);

}  // namespace cb
#endif
