// Index checks of a plan (the stand-in for a memory checker, which this
// library's tests do not run): kernels that read every index array of the
// plan, compare each index with the range the plan's definition (Sec. III-A)
// allows it, and count the ones outside.  They never use an index to
// address memory, so a corrupt plan is reported, not dereferenced.
#include "internal.h"

#include <cuda_runtime.h>

namespace spmvk {

namespace {

// The last i in [0, m) with off[i] <= v (off ascending, off[0] <= v).
__device__ __forceinline__ int find_seg(const int64_t* off, int m, int64_t v) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// CSR rows [0, nrows): ptr ascending within [0, nnz], ptr[0] = 0,
// ptr[nrows] = nnz; the entries of row i, which belongs to group
// g = find_seg(row_off, G, i), lie in [lo[g], hi[g]).
__global__ void check_csr_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, int64_t nrows,
                                 int64_t nnz, const int64_t* __restrict__ row_off, int G,
                                 const int64_t* __restrict__ lo, const int64_t* __restrict__ hi,
                                 unsigned long long* bad) {
    unsigned long long mine = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nrows; i += stride) {
        const int64_t a = ptr[i];
        if (a < 0 || a > nnz) { ++mine; continue; }
        if (i == 0 && a != 0) ++mine;
        if (i == nrows) {
            if (a != nnz) ++mine;
            continue;
        }
        const int64_t b = ptr[i + 1];
        if (b < a || b > nnz) { ++mine; continue; }
        const int g = find_seg(row_off, G, i);
        for (int64_t k = a; k < b; ++k) {
            const int64_t c = col[k];
            if (c < lo[g] || c >= hi[g]) ++mine;
        }
    }
    if (mine) atomicAdd(bad, mine);
}

// idx[k] for k in [0, count), k in segment s = find_seg(seg, S, k), must lie
// in [lo[s], hi[s]).
__global__ void check_list_kernel(const int32_t* __restrict__ idx, int64_t count, const int64_t* __restrict__ seg,
                                  int S, const int64_t* __restrict__ lo, const int64_t* __restrict__ hi,
                                  unsigned long long* bad) {
    unsigned long long mine = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        const int s = find_seg(seg, S, k);
        const int64_t v = idx[k];
        if (v < lo[s] || v >= hi[s]) ++mine;
    }
    if (mine) atomicAdd(bad, mine);
}

// A sliced layout: every slice's slots inside the value array, its positions
// inside [0, npos); per live position a length of at most kSellLong (or the
// long-row mark), a row (through perm) in [0, npos); every live slot's x
// index (xoff + column, or row + delta for the 16-bit form) in [x_lo, x_hi);
// every long-row piece inside its row's CSR entries.
__global__ void check_sell_kernel(const SellSlice* __restrict__ slices, int n_slices, const uint8_t* __restrict__ len,
                                  const int32_t* __restrict__ perm, const int32_t* __restrict__ col,
                                  const int16_t* __restrict__ col16, int64_t entries, int64_t npos, int64_t x_lo,
                                  int64_t x_hi, const SellLong* __restrict__ longs, int n_longs,
                                  const int32_t* __restrict__ csr_ptr, unsigned long long* bad) {
    unsigned long long mine = 0;
    const int lane = threadIdx.x & 31;
    const int nw = (int)(gridDim.x * blockDim.x) >> 5;
    for (int si = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); si < n_slices; si += nw) {
        const SellSlice d = slices[si];
        if (d.len < 0 || d.len > kSellLong || d.rows < 0 || d.rows > 32 || d.p0 < 0 || (int64_t)d.p0 + d.rows > npos ||
            d.off < 0 || (int64_t)d.off + 32 * (int64_t)d.len > entries) {
            if (lane == 0) ++mine;
            continue;
        }
        if (lane >= d.rows) continue;
        const int64_t pos = (int64_t)d.p0 + lane;
        const int code = len[pos];
        if (code == kSellLenLong) continue;
        if (code > d.len) { ++mine; continue; }
        const int64_t row = perm ? (int64_t)perm[pos] : pos;
        if (row < 0 || row >= npos) { ++mine; continue; }
        for (int j = 0; j < code; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            const int64_t xi = col16 ? row + (int64_t)col16[o] : (int64_t)d.xoff + col[o];
            if (xi < x_lo || xi >= x_hi) ++mine;
        }
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_longs; i += stride) {
        const SellLong L = longs[i];
        if (L.row < 0 || L.row >= npos) { ++mine; continue; }
        const int64_t a = csr_ptr[L.row], b = csr_ptr[L.row + 1];
        if (L.k0 < a || L.k1 > b || L.k0 >= L.k1 || L.nparts < 1) ++mine;
    }
    if (mine) atomicAdd(bad, mine);
}

int grid_for(int64_t items, int num_sms) {
    int64_t g = (items + 255) / 256;
    if (g < 1) g = 1;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    return (int)g;
}

}  // namespace

cudaError_t launch_check_csr(const int32_t* ptr, const int32_t* col, int64_t nrows, int64_t nnz,
                             const int64_t* row_off, int G, const int64_t* lo, const int64_t* hi,
                             unsigned long long* bad, int num_sms, cudaStream_t s) {
    check_csr_kernel<<<grid_for(nrows + 1, num_sms), 256, 0, s>>>(ptr, col, nrows, nnz, row_off, G, lo, hi, bad);
    return cudaGetLastError();
}

cudaError_t launch_check_list(const int32_t* idx, int64_t count, const int64_t* seg, int S, const int64_t* lo,
                              const int64_t* hi, unsigned long long* bad, int num_sms, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    check_list_kernel<<<grid_for(count, num_sms), 256, 0, s>>>(idx, count, seg, S, lo, hi, bad);
    return cudaGetLastError();
}

cudaError_t launch_check_sell(const SellSlice* slices, int n_slices, const uint8_t* len, const int32_t* perm,
                              const int32_t* col, const int16_t* col16, int64_t entries, int64_t npos, int64_t x_lo,
                              int64_t x_hi, const SellLong* longs, int n_longs, const int32_t* csr_ptr,
                              unsigned long long* bad, int num_sms, cudaStream_t s) {
    const int64_t items = (int64_t)n_slices * 32 > n_longs ? (int64_t)n_slices * 32 : n_longs;
    if (items <= 0) return cudaSuccess;
    check_sell_kernel<<<grid_for(items, num_sms), 256, 0, s>>>(slices, n_slices, len, perm, col, col16, entries, npos,
                                                               x_lo, x_hi, longs, n_longs, csr_ptr, bad);
    return cudaGetLastError();
}

}  // namespace spmvk
