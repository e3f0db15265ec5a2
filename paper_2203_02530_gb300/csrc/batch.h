// Resident matrix store shared by the batched products and the serving
// runtime (include/spmv.h: spmv_batch_*, spmv_serve_*).
#pragma once

#include "part.h"

#include <vector>

namespace spmvk {

// One matrix of a batch: its row pointers start at ptr_off (values local
// to the matrix), its entries at ent_off (a multiple of 4), and its x / y
// at row_off of the concatenated vectors.
struct BatchMat {
    long long ptr_off;
    long long ent_off;
    long long row_off;
    int n;
    int lanes;
};

struct BatchItem;

}  // namespace spmvk

struct spmv_batch {
    int device = 0, num_sms = 0, occupancy = 0;
    int count = 0;
    std::vector<spmvk::BatchMat> mats;   // host copy
    std::vector<int64_t> n;              // rows per matrix
    std::vector<int64_t> nnz;            // entries per matrix
    std::vector<int> item_off;           // count+1 item offsets per matrix
    long long total_rows = 0, total_nnz = 0;
    int32_t* ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    spmvk::BatchMat* d_mats = nullptr;
    void* d_items = nullptr;
    int* ticket = nullptr;
    int n_items = 0;
    size_t device_bytes = 0;
    std::vector<void*> allocs;
};
