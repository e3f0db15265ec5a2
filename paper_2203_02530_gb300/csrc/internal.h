// Internal declarations shared by the host runtime and the kernels of the
// partitioned SpMV library.  Not part of the C ABI (include/spmv.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

namespace spmvk {

// Tile of rows processed by one CTA iteration: rows [r0, r1) of a CSR whose
// entries [k0, k1) are staged in shared memory.  xoff is added to every
// column index before x is read.  flags: TILE_LONG marks a single row longer
// than the stage capacity, summed by the whole CTA straight from global
// memory.
struct Tile {
    int32_t r0, r1, k0, k1;
    int32_t xoff, flags, pad0, pad1;
};
static_assert(sizeof(Tile) == 32, "tile descriptor is two int4");
enum { TILE_LONG = 1 };

// Geometry of the thread-per-row tile kernel.
struct TileGeom {
    int threads;   // threads per CTA
    int nnz_cap;   // entries per tile stage
    int stages;    // shared-memory ring depth
    int chunk;     // x gathers issued together per thread
    int lanes;     // threads per row; a tile holds threads / lanes rows
    int rows() const { return threads / lanes; }
};

// Merge-path tile: merge items [d0, d1) of the (row ends, entries) merge of
// one rank's CSR; (r0, k0) is the path coordinate at d0, (r1, k1) at d1.
struct MergeTile {
    int32_t r0, r1, k0, k1;
    int32_t xoff, pad0, pad1, pad2;
};
static_assert(sizeof(MergeTile) == 32, "merge tile descriptor is two int4");

// Carry of a row cut by a merge tile boundary.
struct Carry {
    int32_t row;   // row index (in the CSR's row space), -1 when none
    int32_t pad;
    double val;
};

// Slice of the sliced-ELL layout: positions [p0, p0 + rows) (rows <= 32) of
// the layout's row order, every row padded to len entries; entry j of lane r
// at off + 32 j + r.
struct SellSlice {
    int32_t p0, rows, len, xoff;
    int32_t off, pad0, pad1, pad2;
};
static_assert(sizeof(SellSlice) == 32, "slice descriptor is two int4");

// A piece of a row longer than kSellLong entries: entries [k0, k1) of the
// CSR row, summed by a whole warp.  A row longer than kSellChunk entries is
// cut into nparts pieces; each writes its partial sum to slot `slot` of the
// partial array, and the warp that finishes a row's last piece (counter
// cidx) adds the row's partials in piece order and stores the row.
struct SellLong {
    int32_t row, xoff, k0, k1;
    int32_t slot, first, nparts, cidx;
};
static_assert(sizeof(SellLong) == 32, "long-row piece is two int4");
constexpr int kSellLong = 64;
constexpr int kSellChunk = 512;
constexpr uint8_t kSellLenLong = 0xFF;   // length code of a long row inside a slice

// Sliced layout of one CSR product (local or remote), all ranks.
struct SellArgs {
    const SellSlice* slices;
    const SellLong* longs;
    const double* val;
    const int32_t* col;
    const int16_t* col16;    // column - row deltas (16-bit variant), or nullptr
    const uint8_t* len;      // per position: entries, or kSellLenLong
    const int32_t* perm;     // per position: row; nullptr = position is the row
    int slice_begin, slice_end, long_begin, long_end;
    double* long_part;       // partial sums of the pieces of cut rows
    int* long_cnt;           // per cut row: pieces done (zero between launches)
    const int32_t* cta_off;  // nullptr: units round-robin over the warps; else
                             // CTA b takes units [cta_off[b], cta_off[b + 1])
    const int32_t* ypos;     // per position: its y row (row order and row map
                             // composed; sorted remote layouts), or nullptr
};

// Operands of one CSR product launch.
struct CsrArgs {
    const int32_t* ptr;     // row pointer of the CSR (row space indices)
    const int32_t* col;
    const double* val;
    const int32_t* rowmap;  // nullptr: output row = row; else y[rowmap[row]]
    const double* x;
    double* y;
    int accumulate;         // 0: y = A x ; 1: y += A x
    int n_rows;             // rows of the CSR row space
    int nnz_total;          // entries of the CSR (bounds the guarded reads)
    int guarded;            // 1: arrays are not padded past their ends
    int* err;               // device error word
    int abort_tile;         // test hook of the merge-path kernel: k > 0 makes
                            // tiles k-1 and later take the path of a wait that
                            // ran out (after their copies landed); 0 = never
    int pdl;                // programmatic-launch flags of the launch
                            // (kPdlNoWait, kPdlEarly; 0 = wait, no early release)
};

// Launchers (kernels.cu).  All return cudaGetLastError() after the launch.
cudaError_t launch_gather(const double* x, const int32_t* idx, const int32_t* pos,
                          double* dst, int64_t count, int num_sms, cudaStream_t s, int pdl = 0);
cudaError_t launch_copy(const double* src, double* dst, int64_t count, int num_sms,
                        cudaStream_t s, int pdl = 0);
cudaError_t launch_tile(const CsrArgs& a, const Tile* tiles, int tile_begin,
                        int tile_end, const TileGeom& g, int num_sms, cudaStream_t s);
cudaError_t launch_vector(const CsrArgs& a, const Tile* tiles, int tile_begin, int tile_end,
                          int lanes, int num_sms, cudaStream_t s);
cudaError_t launch_warp(const CsrArgs& a, const Tile* tiles, int tile_begin, int tile_end,
                        int param, int num_sms, cudaStream_t s);
int warp_tile_cap(int param);
cudaError_t selftest_wait_timeout(uint64_t limit_ns, int* status_host);
int probe_threads();
cudaError_t launch_dfma_probe(int64_t iters, int grid, int lanes, double* out, int64_t* dfma, cudaStream_t s);
cudaError_t launch_gather_probe(const double* table, const int32_t* idx, int64_t count, int grid, double* out,
                                cudaStream_t s);
cudaError_t launch_pairs(const CsrArgs& a, const Tile* tiles, int tile_begin, int tile_end,
                         int lanes, int num_sms, cudaStream_t s);
cudaError_t launch_merge(const CsrArgs& a, const MergeTile* tiles, int tile_begin,
                         int tile_end, Carry* carries, int num_sms, cudaStream_t s);
cudaError_t launch_merge_partition(const int32_t* ptr, int row_begin, int row_end, int32_t xoff,
                                   MergeTile* tiles, int n_tiles, cudaStream_t s);
int merge_items_per_tile();
cudaError_t read_clear_csr_error(int* out);
int64_t noalloc_max_items();
cudaError_t launch_merge_noalloc(const CsrArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_sell_fill(const int32_t* ptr, const int32_t* col, const double* val, const SellSlice* slices,
                             int n_slices, const uint8_t* len, const int32_t* perm, double* sval, int32_t* scol,
                             int num_sms, cudaStream_t s);
cudaError_t launch_sell(const CsrArgs& a, const SellArgs& s, int param, bool delta16, int num_sms,
                        cudaStream_t st);
cudaError_t launch_sell_delta(const SellSlice* slices, int n_slices, const uint8_t* len, const int32_t* perm,
                              const int32_t* scol, int16_t* scol16, int* bad, int num_sms, cudaStream_t s);
bool sell_param_supported(int param);
cudaError_t launch_segment_copy(const int32_t* tab, int n_seg, const double* sv, const int32_t* sc, double* dv,
                                int32_t* dc, int num_sms, cudaStream_t s);
cudaError_t launch_sell_unfill(const int32_t* ptr, const SellSlice* slices, int n_slices, const uint8_t* len,
                               const int32_t* perm, const double* sval, const int32_t* scol, const int16_t* scol16,
                               int32_t* col, double* val, int num_sms, cudaStream_t s);
cudaError_t launch_sell_col32(const SellSlice* slices, int n_slices, const uint8_t* len, const int32_t* perm,
                              const int16_t* scol16, int32_t* scol, int num_sms, cudaStream_t s);

// Index checks (check.cu): count into *bad the indices outside their ranges;
// read-only, no index is used as an address.
cudaError_t launch_check_csr(const int32_t* ptr, const int32_t* col, int64_t nrows, int64_t nnz,
                             const int64_t* row_off, int G, const int64_t* lo, const int64_t* hi,
                             unsigned long long* bad, int num_sms, cudaStream_t s);
cudaError_t launch_check_list(const int32_t* idx, int64_t count, const int64_t* seg, int S, const int64_t* lo,
                              const int64_t* hi, unsigned long long* bad, int num_sms, cudaStream_t s);
cudaError_t launch_check_sell(const SellSlice* slices, int n_slices, const uint8_t* len, const int32_t* perm,
                              const int32_t* col, const int16_t* col16, int64_t entries, int64_t npos, int64_t x_lo,
                              int64_t x_hi, const SellLong* longs, int n_longs, const int32_t* csr_ptr,
                              unsigned long long* bad, int num_sms, cudaStream_t s);
// Params 2000 + p: the launch of param p with cost-balanced contiguous CTA
// ranges (SellArgs::cta_off) instead of the round-robin split.
inline bool sell_param_balanced(int param) { return param >= 2000; }
// CTAs of a sliced launch of `units` work units.
int sell_grid(int param, int units, int num_sms);
int tile_ctas_per_sm(const TileGeom& g);
bool tile_geom_supported(const TileGeom& g);
TileGeom default_tile_geom();

}  // namespace spmvk
