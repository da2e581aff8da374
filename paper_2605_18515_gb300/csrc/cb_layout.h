// Device-resident layout of an analysed matrix, shared by the host analyser (analyze.cpp)
// and the kernels (kernels.cu). Plain structs, no CUDA or C++ library types.
//
// Packed sub-block stream (Sec. 3.2, "intra-block data aggregation"): every non-empty
// 16x16 sub-block ("tile") occupies one 16-byte aligned record of the byte stream; its
// virtual pointer is the record's offset in 16-byte units. Inside a record:
//   COO   (nnz < th1):  nnz coordinate bytes (row = b & 15, col = b >> 4; Sec. 3.2 and the
//                       decode of Algorithm 3), entries sorted by (row, col);
//                       zero padding to 16 B; nnz values.
//   CSR   (otherwise):  17 row-pointer bytes (0..nnz), then the same coordinate bytes,
//                       padding to 16 B, nnz values.
//   DENSE (nnz > th2):  a 32-byte presence bitmap (bit r*16+c), then 256 values
//                       row-major (Algorithm 4 reads dense_val[row*16 + col]); absent
//                       entries hold +0.0. The bitmap keeps explicitly stored zeros
//                       distinguishable so the CSR round trip is exact; the kernel
//                       ignores it.
// Values are stored in the handle's value type; the record size is rounded up to 16 B.
//
// Column aggregation (Sec. 3.3.1): when on, tile column c of a tile with x-base xb reads
// x[restore_cols[xb + c]]; when off, x[xb + c] (xb = 16 * block column).
#ifndef CB_LAYOUT_H_
#define CB_LAYOUT_H_
#include <stdint.h>

#define CB_BLK 16
#define CB_FMT_COO 0
#define CB_FMT_CSR 1
#define CB_FMT_DENSE 2

// One high-level metadata record per tile (the five arrays of Sec. 3.1, minus the
// block column which the kernel does not need, plus the x base it does need).
struct CbTile {
  uint32_t vp16;    // virtual pointer: byte offset of the record / 16
  uint32_t xbase;   // restore_cols index (aggregated) or first column (plain) of column 0
  uint32_t brow;    // block row
  uint16_t nnz;     // stored entries (1..256)
  uint8_t fmt;      // CB_FMT_*
  uint8_t pad;
};

// A unit of work: a run of consecutive tiles processed by one warp. Either a group of
// whole block rows [brow_lo, brow_lo + nbr) (split < 0), or one part of a single block
// row that was cut into nparts units (split >= 0); the parts combine through the
// partial-sum buffer in a fixed order.
struct CbUnit {
  uint32_t tile_lo;   // first tile
  uint16_t ntiles;
  uint16_t nbr;       // block rows covered (1 for split parts)
  uint32_t brow_lo;
  uint32_t byte_lo16; // stream offset of the first tile / 16
  uint32_t nbytes;    // stream bytes of the unit's tiles (multiple of 16)
  uint32_t work;      // multiply-adds: sum of nnz (COO/CSR) and 256 per Dense tile
  uint32_t rc_lo;     // first restore_cols entry copied (multiple of 4)
  uint32_t rc_n;      // restore_cols entries copied (multiple of 4; 0 when plain)
  int32_t split;      // split-row id or -1
  uint16_t part, nparts;
  uint32_t slot;      // partial-sum slot of this part (16 values per slot)
  uint32_t sched16;   // offset of the unit's lane schedule in the schedule array / 16
  uint32_t sched_bytes;  // bytes of the schedule (multiple of 16)
  uint32_t blob16;    // offset of the unit blob in the blob array / 16
  uint32_t blob_bytes;   // 16 * ntiles + 4 * rc_n + sched_bytes
  uint32_t mode;         // CB_MODE_* flags of the unit's lane schedule
};
#define CB_MODE_ENTRY 1u     // schedule of single entries instead of chunks of up to CB_CHUNK
#define CB_MODE_SCAN 2u      // some row spans more than CB_SCAN_SPAN lanes: resolve carries by a scan
#define CB_MODE_XSEQ 4u      // every chunk covers consecutive columns of its tile (pieces cut at
                             // column gaps): one coordinate byte and contiguous x per chunk
#define CB_MODE_DIRECT 8u    // (with ENTRY or XSEQ) 32-bit chunk descriptors that hold the
                             // chunk's value offset and first column (layout below)
#define CB_SCAN_SPAN 4

// Unit blob: the unit's tile records, its restore_cols slice and its lane schedule, stored
// back to back (each part a multiple of 16 bytes) so that the kernel stages all of the
// unit's metadata with one bulk copy:
//   [0, 16 * ntiles) tile records | [.., + 4 * rc_n) restore_cols | [.., + sched_bytes) schedule

// A block row cut into several units: its parts store 16 partial row sums each in
// consecutive slots slot0 .. slot0 + nparts - 1; a second kernel adds them in a fixed order.
// Rows with more than CB_COMBINE_WIDE_PARTS parts are stored last and added by 16 lanes
// per row instead of one.
#define CB_COMBINE_WIDE_PARTS 16
struct CbSplitRow {
  uint32_t slot0;
  uint32_t brow;
  uint16_t nparts;
  uint16_t rows;      // rows of the block row inside the matrix (<= 16)
  uint32_t pad;
};

// Lane schedule of a unit (built by the analyser, staged with the unit). The unit's
// multiply-adds are taken in row-major order (row, then tile, then entry) and cut into
// chunks of at most CB_CHUNK consecutive entries of one (tile, row) piece (single entries
// in CB_MODE_ENTRY units; chunks also end at column gaps in CB_MODE_XSEQ units); the chunk
// list is dealt to CB_VLANES runs of (nearly) equal length, one per lane. A lane takes its
// run's chunks two at a time (chunk A, chunk B) into one accumulator per vector.
// Layout:
//   CB_VLANES x uint16 run header: bits [0,8) row of the run's first chunk, bit 8 set when
//     that row began in an earlier run, bits [9,16) number of chunks of the run;
//   R x uint8 next row: for each row of the unit, the next row holding entries;
//   padding to a multiple of 16 bytes from the start;
//   rows / 2 x CB_VLANES x uint32 chunk-descriptor pairs, row-major by (pair index, run):
//   the low half holds chunk 2i of the run, the high half chunk 2i + 1; rows = the longest
//   run's chunk count rounded up to an even number. A 16-bit chunk descriptor:
//     bits [0,5) tile in the unit, [5,13) first entry inside the tile record (entry order
//     of the record: row-major; Dense: row * 16 + col), [13,15) length 1..CB_CHUNK (0 = no
//     chunk), bit 15 set when the chunk ends its row.
//   CB_MODE_DIRECT units (single-entry or consecutive-column chunks; at most
//   CB_DIRECT_MAX_CHUNKS chunks) instead hold rows / 2 x CB_VLANES x (2 x uint32) pairs of
//   32-bit direct descriptors: bits [0,12) byte offset / 2 of the chunk's first value from
//   the start of the unit's stream bytes, [12,17) tile in the unit, [17,21) column of the
//   first entry in the tile, [21,23) length (0 = no chunk), bit 23 set when the chunk ends
//   its row, [24,32) first entry inside the tile record. The run kernel then needs neither
//   the tile bases nor the coordinate bytes to find a chunk's values and x values. A direct
//   unit's stream bytes hold its tiles' coordinate parts (index bytes, CSR row pointer or
//   Dense bitmap; 16-byte aligned, tile order) followed by its values in load order: for
//   each chunk index j within a run, the chunks j of lanes 0..31, each chunk's values
//   consecutive.
#define CB_CHUNK 3
// A unit whose chunks of up to CB_CHUNK entries would fill less than this share of their
// FMA slots (sparse tiles, rows with one or two entries per tile) is scheduled in single
// entries instead (mode 1): fewer wasted FMA slots and loads per entry.
#ifndef CB_ENTRY_MODE_FILL
#define CB_ENTRY_MODE_FILL 0.6
#endif
#define CB_VLANES 32
#define CB_DIRECT_MAX_CHUNKS 512   // direct descriptors: 16 rows of 32 lanes x 4 bytes fit the
                                   // schedule space of 32 rows x 2 bytes
#define CB_SCHED_HDR(R) ((2u * CB_VLANES + (uint32_t)(R) + 15u) & ~15u)
#define CB_STEPS_MAX ((((CB_UNIT_WORK_MAX + CB_VLANES - 1) / CB_VLANES) + 1) & ~1)
#define CB_SCHED_MAX (CB_SCHED_HDR(CB_R_MAX) + 2 * CB_VLANES * CB_STEPS_MAX)

// Limits the analyser must respect when it cuts units: every unit must fit one warp buffer
// of the run kernel, so they also set how many worker warps fit an SM (FP64 14, FP32 22,
// BF16/FP16 24). Each was chosen by timing the FEM and R-MAT workloads over a few sizes
// and can be overridden at compile time for such sweeps.
#ifndef CB_B_MAX
#define CB_B_MAX 8192           // stream bytes per unit, 8-byte values
#endif
#ifndef CB_B_MAX_4
#define CB_B_MAX_4 4096         // stream bytes per unit, 4-byte values
#endif
#ifndef CB_B_MAX_2
#define CB_B_MAX_2 3072         // stream bytes per unit, 2-byte values
#endif
#define CB_B_MAX_FOR(vsize) ((vsize) == 8 ? CB_B_MAX : (vsize) == 4 ? CB_B_MAX_4 : CB_B_MAX_2)
#ifndef CB_T_MAX
#define CB_T_MAX 20             // tiles per unit (at most 32: 5-bit tile field of a descriptor)
#endif
#define CB_NBR_MAX 8            // block rows per group unit
#define CB_R_MAX (CB_NBR_MAX * CB_BLK)
#define CB_RC_MAX (CB_T_MAX * 16 + 16)   // restore_cols entries per unit (incl. alignment)
#define CB_RC_PAD 32            // zero entries appended to restore_cols
#ifndef CB_UNIT_WORK_DEFAULT
#define CB_UNIT_WORK_DEFAULT 1024
#endif
#ifndef CB_UNIT_WORK_MAX
#define CB_UNIT_WORK_MAX 1024   // multiply-adds per unit (bounds the chunks per unit)
#endif

// ---- Lane-stream layout (FP64 values; every value type with record_layout 2) -------------
// On GB300 a warp-wide FP64 FMA holds its SM sub-partition's FP64 pipe for 76 cycles (the
// pipe retires 32 lanes in that time whether they are active or not), so the FP64 kernel's
// bound is the number of FMA slots it issues, and every issue slot not spent on a useful
// FMA, or spent waiting for an operand, is lost. For FP64 values the analysis therefore
// packs each unit's sub-blocks (intra-block data aggregation, Sec. 3.2, applied to the
// unit's group of sub-blocks) behind the unit's virtual pointers in the order the warp
// consumes them: the unit's stored entries, taken row by row (row, then sub-block, then
// column), are dealt to the 32 lanes in runs of (nearly) equal length; step s of lane l is
// entry c0(l) + s, c0(l) = floor(l * W / 32), W = the unit's entries.
//   values, FP64: steps x 32 doubles, step-major (one coalesced 256-byte load per step);
//           absent entries (past a lane's run) hold +0.0.
//   values, FP32 / BF16 / FP16: full groups of 8 steps, per group 32 lanes x 8 values,
//           each lane's 8 steps contiguous (one 16-byte load per lane and group for the
//           2-byte types, two for FP32); then the last t = steps mod 8 steps (if any) as
//           32 lanes x t values, each lane's t contiguous (no padding to a full group);
//           absent entries hold +0.
//   words, FP64: ceil(steps / 4) x 32 x uint64, each the four 16-bit entry words of steps
//           4q .. 4q + 3 of one lane: bits [0, 9) x slot of the entry (16 * sub-block in
//           the unit + column in the sub-block, the coordinate nibble of Sec. 3.2),
//           bits [9, 16) row in the unit (16 * block row in the unit + row nibble; a
//           unit holds at most 7 block rows, so a word of an entry is below 0xe000);
//           0xffff = no entry.
//   words, FP32 / BF16 / FP16: per full group of 8 steps 32 lanes x 2 uint64 (steps
//           8g .. 8g+3, then 8g+4 .. 8g+7), the same 16-bit entry words; the last t steps:
//           32 lanes x ceil(t / 4) uint64.
//   gather list, aggregated units: 16 per sub-block of the unit, the x column of every x
//           slot (restore_cols[xbase + c]), -1 for slots past the block row's kept columns.
//           When the unit's columns span fewer than 65,535 values (CB_LUNIT_G16), the
//           same list as uint16 offsets from the unit's first column (gbase), 0xffff for
//           -1, in the first half of the list's 32-bit space (half the bytes to read).
//   gather list, plain units (CB_LUNIT_PLAINX, no aggregation): one per sub-block, its
//           first column 16 * block column; slot 16 t + c reads x[gcols[t] + c] (zero at or
//           past n). Padded to a multiple of 4 entries (16 bytes).
// Every format keeps its stored entries only: Dense zero fill (Algorithm 4) would cost a
// full FP64 FMA slot per zero. The sub-block records, formats and restore_cols stay the
// analysis result (export_blocked, statistics); the record stream is not uploaded.
#define CB_LANE_T_MAX 32             // sub-blocks per unit: 512 x slots (the 9-bit slot field)
#define CB_LANE_SLOTS (16 * CB_LANE_T_MAX)
#define CB_LANE_WORK_DEFAULT 2048    // target stored entries per unit
#define CB_LANE_WORK_MAX 16384
#define CB_LANE_NBR_MAX 7            // block rows per unit: rows <= 111, so no entry word is 0xffff
#define CB_LANE_NONE 0xffffu
#define CB_LUNIT_SCAN 1u             // some row spans more than CB_SCAN_SPAN lanes
#define CB_LUNIT_PLAINX 2u           // plain sub-blocks: one gather-list entry per sub-block
#define CB_LUNIT_G16 4u              // per-slot gather list as uint16 offsets from gbase
#define CB_LANE_GROUP 8              // steps per group of the reduced-type layout

#ifdef __CUDACC__
#define CB_LAYOUT_HD __host__ __device__
#else
#define CB_LAYOUT_HD
#endif
// Element index, from the unit's first value (vals * 32), of step st of lane l in a unit of
// S steps; grouped: the reduced-type layout.
CB_LAYOUT_HD inline uint32_t cb_lane_val_index(bool grouped, uint32_t st, uint32_t l, uint32_t S) {
  if (!grouped) return st * CB_VLANES + l;
  const uint32_t full = S / CB_LANE_GROUP * CB_LANE_GROUP;   // steps in full groups
  if (st < full) return (st / CB_LANE_GROUP) * (CB_LANE_GROUP * CB_VLANES) + l * CB_LANE_GROUP + st % CB_LANE_GROUP;
  return full * CB_VLANES + l * (S - full) + (st - full);
}
// uint64 index, from the unit's first word row (words * 32), of the word holding step st of
// lane l (at bit 16 * (st % 4)) in a unit of S steps.
CB_LAYOUT_HD inline uint32_t cb_lane_word_index(bool grouped, uint32_t st, uint32_t l, uint32_t S) {
  if (!grouped) return (st / 4) * CB_VLANES + l;
  const uint32_t full = S / CB_LANE_GROUP * CB_LANE_GROUP;
  if (st < full) return (st / CB_LANE_GROUP) * (2 * CB_VLANES) + 2 * l + (st % CB_LANE_GROUP) / 4;
  return (full / 4) * CB_VLANES + l * ((S - full + 3) / 4) + (st - full) / 4;
}
struct CbLaneUnit {                  // 32 bytes
  uint32_t vals;        // first step of the unit's values (in steps of 32 values)
  uint32_t words;       // first word row (in rows of 32 uint64)
  uint32_t gcols;       // first gather-list entry
  uint32_t brow_lo;     // first block row
  uint16_t steps;       // steps per lane (ceil(W / 32))
  uint16_t nslots;      // x slots (16 * sub-blocks)
  uint16_t nrows;       // rows of the unit inside the matrix (<= 128)
  uint16_t flags;       // CB_LUNIT_*
  uint32_t slot;        // partial-sum slot of a block-row part, 0xffffffff for whole block rows
  uint32_t gbase;       // CB_LUNIT_G16: column that the uint16 gather offsets start from
};

#endif
