// Resident matrix store shared by the batched products and the serving
// runtime (include/spmv.h: spmv_batch_*, spmv_serve_*).
#pragma once

#include "part.h"

#include <vector>

namespace spmvk {

// Slice of a matrix's sliced layout: positions [pos0, pos0 + rows) of the
// matrix's row order, entry j of lane r at off + 32 j + r, len slots each.
struct BSlice {
    int32_t pos0, rows, len, off;
};

// One matrix of a batch: its row pointers start at ptr_off (values local
// to the matrix), its entries at ent_off (a multiple of 4), and its x / y
// at row_off of the concatenated vectors.  The s_* arrays hold its sliced
// layout once built (lanes == 64): row order s_perm (nullptr = natural),
// the first n_long positions are rows summed by a whole warp, the rest
// (lengths s_len) are cut into n_slices slices.
struct BatchMat {
    long long ptr_off;
    long long ent_off;
    long long row_off;
    int n;
    int lanes;
    const double* s_val;
    const int32_t* s_col;
    const uint8_t* s_len;
    const int32_t* s_perm;
    const BSlice* s_slices;
    int n_long;
    int n_slices;
    int n_vlong;   // of the long rows, the first n_vlong are longer than 2048
                   // entries (served by a whole CTA each)
    int pad;
};

// Work item: kind 0 = rows [a, b) in CSR form; kind 1 = positions [a, b)
// of long rows (sliced layout); kind 2 = slices [a, b) (sliced layout).
struct BatchItem {
    int m, kind, a, b;
};

}  // namespace spmvk

struct spmv_batch {
    int device = 0, num_sms = 0, occupancy = 0, occupancy_sliced = 0;
    int n_sliced_items = 0;              // leading entries of `order` that are sliced-layout items
    int count = 0;
    std::vector<spmvk::BatchMat> mats;   // host copy
    std::vector<int64_t> n;              // rows per matrix
    std::vector<int64_t> nnz;            // entries per matrix
    std::vector<int> item_off;           // count+1 item offsets per matrix
    std::vector<std::vector<spmvk::BatchItem>> csr_items, sliced_items;   // per matrix
    std::vector<std::vector<int64_t>> csr_cost, sliced_cost;              // estimated work per item
    std::vector<int> order;              // claim order of the persistent launch
    std::vector<char> sliced_built;      // per matrix
    int* d_order = nullptr;
    int* d_order_full = nullptr;         // claim order of a whole-batch launch (sliced items interleaved)
    size_t items_cap = 0;                // capacity of d_items / d_order (items)
    long long total_rows = 0, total_nnz = 0;
    int32_t* ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    spmvk::BatchMat* d_mats = nullptr;
    void* d_items = nullptr;
    int* ticket = nullptr;
    double* io_x = nullptr;              // device vectors of the host-buffer path (built on first use)
    double* io_y = nullptr;
    double* io_x2 = nullptr;             // the second pair of the streamed host-buffer path
    double* io_y2 = nullptr;
    std::vector<cudaEvent_t> io_ev;      // per chunk (64): x arrived, y computed; then x free, y free per pair
    int* io_tickets = nullptr;           // per chunk: a ticket per layout (4 ints)
    std::vector<int> order_off;          // 2 x (count+1): start of matrix m's items in each part of `order`
    int n_items = 0;
    size_t device_bytes = 0;
    std::vector<void*> allocs;
    // CSR released (spmv_batch_release_csr): ptr/col/val then hold only the
    // long rows (shorter rows have zero length); the full row pointers and
    // entry offsets are kept on the host for the rebuild
    bool csr_released = false;
    std::vector<int32_t> h_full_ptr;
    std::vector<long long> full_ent_off;
    long long full_entries = 0;
};
