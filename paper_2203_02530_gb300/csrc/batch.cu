// Many independent CSR products in one persistent launch.
//
// The matrices of a batch live back to back in HBM (row pointers local to
// each matrix, entries padded to a multiple of 4 so every matrix starts
// 16-byte aligned).  A work item is a block of up to 256 rows of one matrix;
// the warps of a persistent grid claim items with an atomic ticket and
// compute every row with the pair-per-lane scheme or warp-staged rows
// (chosen per matrix by the autotuner); rows longer than 64 entries are
// summed by a whole warp.  The plain alternative launches the same per-row
// code once per matrix; both give bit-identical results because each row
// is summed by the same lanes in the same order.
#include "batch.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

using spmvk::BatchMat;

namespace {

constexpr int kItemRows = 256;
constexpr int kThreads = 256;

struct BatchItem {
    int m, r0, r1, pad;
};

struct BatchArgs {
    const int32_t* ptr;
    const int32_t* col;
    const double* val;
    const BatchMat* mats;
    const BatchItem* items;
    const double* x;
    double* y;
    int n_items;
    int* ticket;
};

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double ldg_keep(const double* p, uint64_t policy) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(policy));
    return v;
}

constexpr int kLongRow = 64;   // rows longer than this are summed by a whole warp

// One row summed by the 32 lanes of a warp: lane l takes entries l, l+32,
// ... in order (four loads in flight), then a fixed xor-butterfly; every
// lane returns the total.
__device__ __forceinline__ double warp_row(const int32_t* col, const double* val, const double* x, int kb, int ke,
                                           uint64_t pol) {
    const int lane = threadIdx.x & 31;
    double part = 0.0;
    int k = kb + lane;
    for (; k + 96 < ke; k += 128) {
        double v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            v[u] = __ldg(val + k + 32 * u);
            xv[u] = ldg_keep(x + __ldg(col + k + 32 * u), pol);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) part = fma(v[u], xv[u], part);
    }
    for (; k < ke; k += 32) part = fma(__ldg(val + k), ldg_keep(x + __ldg(col + k), pol), part);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    return part;
}

// The long rows flagged in `mask` (bit = the lane holding the row's kb, ke
// and row index), one after another, each by the whole warp.
__device__ __forceinline__ void warp_long_rows(unsigned mask, int kb, int ke, int row, const int32_t* col,
                                               const double* val, const double* x, double* y, uint64_t pol) {
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const int rkb = __shfl_sync(0xffffffffu, kb, src);
        const int rke = __shfl_sync(0xffffffffu, ke, src);
        const int rrow = __shfl_sync(0xffffffffu, row, src);
        const double t = warp_row(col, val, x, rkb, rke, pol);
        if ((threadIdx.x & 31) == 0) y[rrow] = t;
    }
}

// Rows [r0, r1) of one matrix by one warp: V lanes per row, lane h takes the
// aligned entry pairs h, h+V, ...; the FMA loop runs the warp's longest
// share.  Rows longer than kLongRow are left out of that loop and summed
// afterwards by the whole warp, so one long row never holds 32 / V short
// ones (or the warp) for its whole length.
template <int V>
__device__ __forceinline__ void batch_rows(const BatchArgs& a, const BatchMat& m, int r0, int r1, uint64_t pol) {
    constexpr int GROUPS = 32 / V;
    constexpr int U = 4;
    const int lane = (threadIdx.x & 31) % V;
    const int group = (threadIdx.x & 31) / V;
    const int32_t* ptr = a.ptr + m.ptr_off;
    const int32_t* col = a.col + m.ent_off;
    const double* val = a.val + m.ent_off;
    const double* x = a.x + m.row_off;
    double* y = a.y + m.row_off;
    for (int rbase = r0; rbase < r1; rbase += GROUPS) {
        const int row = rbase + group;
        int kb = 0, ke = 0, k2 = 0, cnt = 0;
        bool is_long = false;
        if (row < r1) {
            kb = __ldg(ptr + row);
            ke = __ldg(ptr + row + 1);
            is_long = V < 32 && ke - kb > kLongRow;
            k2 = kb & ~1;
            const int npairs = (ke - k2 + 1) >> 1;
            cnt = (!is_long && npairs > lane) ? (npairs - lane + V - 1) / V : 0;
        }
        const unsigned long_mask = __ballot_sync(0xffffffffu, is_long && lane == 0);
        const int wmax = __reduce_max_sync(0xffffffffu, cnt);
        double sum = 0.0;
        for (int j0 = 0; j0 < wmax; j0 += U) {
            double2 vv[U];
            double x0[U], x1[U];
            bool m0[U], m1[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                const bool act = j < cnt;
                const int k = act ? k2 + 2 * (lane + V * j) : k2;
                vv[u] = __ldg(reinterpret_cast<const double2*>(val + k));
                const int2 c = __ldg(reinterpret_cast<const int2*>(col + k));
                m0[u] = act && k >= kb;
                m1[u] = act && k + 1 < ke;
                x0[u] = ldg_keep(x + (m0[u] ? c.x : 0), pol);
                x1[u] = ldg_keep(x + (m1[u] ? c.y : 0), pol);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j0 + u >= wmax) break;
                double t = fma(vv[u].x, x0[u], sum);
                sum = m0[u] ? t : sum;
                t = fma(vv[u].y, x1[u], sum);
                sum = m1[u] ? t : sum;
            }
        }
#pragma unroll
        for (int off = V / 2; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off, V);
        if (row < r1 && lane == 0 && !is_long) y[row] = sum;
        warp_long_rows(long_mask, kb, ke, row, col, val, x, y, pol);
    }
}

constexpr int kStageEntries = 448;   // per warp: 32 rows x 14 entries

// Warp-staged rows (lanes = 0), 32 rows per pass: when the pass's short
// rows fit the warp's shared-memory slice, the warp copies their entries in
// with coalesced loads and every lane sums one row from shared memory (one
// DFMA per entry, the FMA loop running the warp's longest short row);
// otherwise each lane sums its short row straight from global memory.
// Rows longer than kLongRow are summed afterwards by the whole warp.
__device__ __forceinline__ void batch_rows_staged(const BatchArgs& a, const BatchMat& m, int r0, int r1,
                                                  uint64_t pol, double* sv, int32_t* sc) {
    constexpr int CH = 8;
    const int lane = threadIdx.x & 31;
    const int32_t* ptr = a.ptr + m.ptr_off;
    const int32_t* col = a.col + m.ent_off;
    const double* val = a.val + m.ent_off;
    const double* x = a.x + m.row_off;
    double* y = a.y + m.row_off;
    for (int rb = r0; rb < r1; rb += 32) {
        const int re = rb + 32 < r1 ? rb + 32 : r1;
        const int k0 = __ldg(ptr + rb), k1 = __ldg(ptr + re);
        const int row = rb + lane;
        int kb = 0, ke = 0;
        if (row < re) {
            kb = __ldg(ptr + row);
            ke = __ldg(ptr + row + 1);
        }
        const bool is_long = ke - kb > kLongRow;
        const unsigned long_mask = __ballot_sync(0xffffffffu, is_long);
        const int cnt = is_long ? 0 : ke - kb;
        const int wmax = __reduce_max_sync(0xffffffffu, cnt);
        double sum = 0.0;
        if (long_mask == 0 && k1 - k0 <= kStageEntries) {
            for (int i = lane; i < k1 - k0; i += 32) {
                sv[i] = __ldg(val + k0 + i);
                sc[i] = __ldg(col + k0 + i);
            }
            __syncwarp();
            const int sb = kb - k0;
            for (int base = 0; base < wmax; base += CH) {
                double xv[CH], vv[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const bool on = base + u < cnt;
                    vv[u] = on ? sv[sb + base + u] : 0.0;
                    xv[u] = ldg_keep(x + (on ? sc[sb + base + u] : 0), pol);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (base + u >= wmax) break;
                    const double t = fma(vv[u], xv[u], sum);
                    sum = base + u < cnt ? t : sum;
                }
            }
            __syncwarp();
        } else {
            for (int base = 0; base < wmax; base += CH) {
                double xv[CH], vv[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const bool on = base + u < cnt;
                    const int k = on ? kb + base + u : 0;
                    vv[u] = on ? __ldg(val + k) : 0.0;
                    xv[u] = ldg_keep(x + (on ? __ldg(col + k) : 0), pol);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (base + u >= wmax) break;
                    const double t = fma(vv[u], xv[u], sum);
                    sum = base + u < cnt ? t : sum;
                }
            }
        }
        if (row < re && !is_long) y[row] = sum;
        warp_long_rows(long_mask, kb, ke, row, col, val, x, y, pol);
    }
}

__device__ __forceinline__ void batch_item(const BatchArgs& a, int it, uint64_t pol, double* sv,
                                           int32_t* sc) {
    const BatchItem w = a.items[it];
    const BatchMat m = a.mats[w.m];
    switch (m.lanes) {
        case 0: batch_rows_staged(a, m, w.r0, w.r1, pol, sv, sc); break;
        case 1: batch_rows<1>(a, m, w.r0, w.r1, pol); break;
        case 2: batch_rows<2>(a, m, w.r0, w.r1, pol); break;
        case 4: batch_rows<4>(a, m, w.r0, w.r1, pol); break;
        case 8: batch_rows<8>(a, m, w.r0, w.r1, pol); break;
        case 16: batch_rows<16>(a, m, w.r0, w.r1, pol); break;
        default: batch_rows<32>(a, m, w.r0, w.r1, pol); break;
    }
}

// Persistent: every warp claims whole items with an atomic ticket until
// none is left (no block-wide barrier: warps never wait for each other).
__global__ void __launch_bounds__(kThreads, 4) batch_persistent_kernel(BatchArgs a) {
    __shared__ double s_val[kThreads / 32][kStageEntries];
    __shared__ int32_t s_col[kThreads / 32][kStageEntries];
    const uint64_t pol = policy_evict_last();
    const int w = threadIdx.x >> 5;
    for (;;) {
        int it = 0;
        if ((threadIdx.x & 31) == 0) it = atomicAdd(a.ticket, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.n_items) break;
        batch_item(a, it, pol, s_val[w], s_col[w]);
    }
}

// Items [first, last), one per warp, grid-stride (one matrix per launch).
__global__ void __launch_bounds__(kThreads, 4) batch_range_kernel(BatchArgs a, int first, int last) {
    __shared__ double s_val[kThreads / 32][kStageEntries];
    __shared__ int32_t s_col[kThreads / 32][kStageEntries];
    const uint64_t pol = policy_evict_last();
    const int w = threadIdx.x >> 5;
    const int nw = (int)gridDim.x * (kThreads / 32);
    for (int it = first + (int)blockIdx.x * (kThreads / 32) + w; it < last; it += nw)
        batch_item(a, it, pol, s_val[w], s_col[w]);
}

}  // namespace

namespace {

int bfail(int code, const std::string& m) {
    spmvk::set_last_error(m);
    return code;
}

void* balloc(spmv_batch* b, size_t bytes) {
    void* p = nullptr;
    spmvk::check_cuda(cudaMalloc(&p, bytes + 256), "cudaMalloc");
    b->allocs.push_back(p);
    b->device_bytes += bytes + 256;
    spmvk::check_cuda(cudaMemset(p, 0, bytes + 256), "cudaMemset");
    return p;
}

void bfree(spmv_batch* b) {
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
}

BatchArgs args_of(spmv_batch* b, const double* x, double* y) {
    BatchArgs a{};
    a.ptr = b->ptr;
    a.col = b->col;
    a.val = b->val;
    a.mats = b->d_mats;
    a.items = static_cast<const BatchItem*>(b->d_items);
    a.x = x;
    a.y = y;
    a.n_items = b->n_items;
    a.ticket = b->ticket;
    return a;
}

}  // namespace

#define BATCH_TRY try {
#define BATCH_CATCH                                                             \
    }                                                                           \
    catch (const spmvk::Fail& f) {                                              \
        return bfail(f.code, f.msg);                                            \
    }                                                                           \
    catch (const std::bad_alloc&) {                                             \
        return bfail(SPMV_ENOMEM, "host allocation failed");                    \
    }                                                                           \
    catch (...) {                                                               \
        return bfail(SPMV_EINVAL, "unexpected exception");                      \
    }

extern "C" {

int spmv_batch_create(int count, const int64_t* n, const int64_t* const* row_ptr,
                      const int32_t* const* col_idx, const double* const* vals, spmv_batch** out) {
    if (!out) return bfail(SPMV_EINVAL, "out is NULL");
    *out = nullptr;
    spmv_batch* b = nullptr;
    BATCH_TRY
    if (count < 1) spmvk::fail(SPMV_EINVAL, "count = %d", count);
    if (!n || !row_ptr || !col_idx || !vals) spmvk::fail(SPMV_EINVAL, "NULL array");
    b = new spmv_batch();
    b->count = count;
    spmvk::check_cuda(cudaGetDevice(&b->device), "cudaGetDevice");
    spmvk::check_cuda(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device), "SMs");
    spmvk::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occupancy, batch_persistent_kernel,
                                                                    kThreads, 0),
                      "occupancy");
    long long ptr_total = 0, ent_total = 0, rows_total = 0;
    b->mats.resize(count);
    b->n.resize(count);
    b->nnz.resize(count);
    for (int m = 0; m < count; ++m) {
        if (n[m] < 0 || n[m] >= (int64_t(1) << 31)) spmvk::fail(SPMV_EINVAL, "matrix %d: n = %lld", m, (long long)n[m]);
        if (n[m] > 0 && !row_ptr[m]) spmvk::fail(SPMV_EINVAL, "matrix %d: row_ptr is NULL", m);
        const int64_t base = n[m] > 0 ? row_ptr[m][0] : 0;
        const int64_t z = n[m] > 0 ? row_ptr[m][n[m]] - base : 0;
        for (int64_t i = 0; i < n[m]; ++i)
            if (row_ptr[m][i + 1] < row_ptr[m][i]) spmvk::fail(SPMV_EINVAL, "matrix %d: row_ptr decreases", m);
        if (z >= (int64_t(1) << 31) - 8) spmvk::fail(SPMV_EBOUNDS, "matrix %d: too many entries", m);
        if (z > 0 && (!col_idx[m] || !vals[m])) spmvk::fail(SPMV_EINVAL, "matrix %d: NULL entries", m);
        for (int64_t k = base; k < base + z; ++k)
            if (col_idx[m][k] < 0 || col_idx[m][k] >= n[m]) spmvk::fail(SPMV_EINVAL, "matrix %d: column out of range", m);
        b->n[m] = n[m];
        b->nnz[m] = z;
        b->mats[m] = BatchMat{ptr_total, ent_total, rows_total, (int)n[m], 2};
        ptr_total += n[m] + 1;
        ent_total += (z + 3) & ~int64_t(3);   // keep every matrix 16-byte aligned
        rows_total += n[m];
    }
    b->total_rows = rows_total;
    for (int64_t z : b->nnz) b->total_nnz += z;
    std::vector<int32_t> hptr((size_t)ptr_total);
    std::vector<int32_t> hcol((size_t)ent_total, 0);
    std::vector<double> hval((size_t)ent_total, 0.0);
    std::vector<BatchItem> items;
    b->item_off.assign(count + 1, 0);
    for (int m = 0; m < count; ++m) {
        const BatchMat& M = b->mats[m];
        const int64_t base = n[m] > 0 ? row_ptr[m][0] : 0;
        for (int64_t i = 0; i <= n[m]; ++i)
            hptr[(size_t)(M.ptr_off + i)] = n[m] > 0 ? (int32_t)(row_ptr[m][i] - base) : 0;
        for (int64_t k = 0; k < b->nnz[m]; ++k) {
            hcol[(size_t)(M.ent_off + k)] = col_idx[m][base + k];
            hval[(size_t)(M.ent_off + k)] = vals[m][base + k];
        }
        b->item_off[m] = (int)items.size();
        for (int64_t r = 0; r < n[m]; r += kItemRows)
            items.push_back(BatchItem{m, (int)r, (int)std::min<int64_t>(n[m], r + kItemRows), 0});
    }
    b->item_off[count] = (int)items.size();
    b->n_items = (int)items.size();
    b->ptr = static_cast<int32_t*>(balloc(b, hptr.size() * 4));
    b->col = static_cast<int32_t*>(balloc(b, hcol.size() * 4));
    b->val = static_cast<double*>(balloc(b, hval.size() * 8));
    b->d_mats = static_cast<BatchMat*>(balloc(b, b->mats.size() * sizeof(BatchMat)));
    b->d_items = balloc(b, items.size() * sizeof(BatchItem));
    b->ticket = static_cast<int*>(balloc(b, sizeof(int)));
    spmvk::check_cuda(cudaMemcpy(b->ptr, hptr.data(), hptr.size() * 4, cudaMemcpyHostToDevice), "upload");
    spmvk::check_cuda(cudaMemcpy(b->col, hcol.data(), hcol.size() * 4, cudaMemcpyHostToDevice), "upload");
    spmvk::check_cuda(cudaMemcpy(b->val, hval.data(), hval.size() * 8, cudaMemcpyHostToDevice), "upload");
    spmvk::check_cuda(cudaMemcpy(b->d_mats, b->mats.data(), b->mats.size() * sizeof(BatchMat),
                                 cudaMemcpyHostToDevice), "upload");
    if (!items.empty())
        spmvk::check_cuda(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem),
                                     cudaMemcpyHostToDevice), "upload");
    *out = b;
    b = nullptr;
    return SPMV_OK;
    }
    catch (const spmvk::Fail& f) {
        if (b) { bfree(b); delete b; }
        return bfail(f.code, f.msg);
    }
    catch (...) {
        if (b) { bfree(b); delete b; }
        return bfail(SPMV_ENOMEM, "batch creation failed");
    }
}

int spmv_batch_destroy(spmv_batch* b) {
    if (!b) return SPMV_OK;
    cudaError_t e = cudaDeviceSynchronize();
    bfree(b);
    delete b;
    return e == cudaSuccess ? SPMV_OK : bfail(SPMV_ECUDA, cudaGetErrorString(e));
}

int spmv_batch_set_lanes(spmv_batch* b, int m, int lanes) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    if (m < -1 || m >= b->count) spmvk::fail(SPMV_EINVAL, "matrix %d", m);
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
        spmvk::fail(SPMV_EINVAL, "lanes %d not in {0,1,2,4,8,16,32}", lanes);
    const int lo = m < 0 ? 0 : m, hi = m < 0 ? b->count : m + 1;
    for (int i = lo; i < hi; ++i) b->mats[i].lanes = lanes;
    spmvk::check_cuda(cudaMemcpy(b->d_mats + lo, b->mats.data() + lo, (size_t)(hi - lo) * sizeof(BatchMat),
                                 cudaMemcpyHostToDevice),
                      "lanes");
    BATCH_CATCH
    return SPMV_OK;
}

int spmv_batch_query(const spmv_batch* b, int what, int m, int64_t* out) {
    BATCH_TRY
    if (!b || !out) spmvk::fail(SPMV_EINVAL, "NULL argument");
    const bool mat = m >= 0 && m < b->count;
    switch (what) {
        case SPMV_BQ_COUNT: *out = b->count; break;
        case SPMV_BQ_DEVICE_BYTES: *out = (int64_t)b->device_bytes; break;
        case SPMV_BQ_TOTAL_ROWS: *out = b->total_rows; break;
        case SPMV_BQ_TOTAL_NNZ: *out = b->total_nnz; break;
        case SPMV_BQ_ITEMS: *out = b->n_items; break;
        case SPMV_BQ_ALG_BYTES:
            // entries, row pointers, x read, y written, over every matrix
            *out = 12 * b->total_nnz + 4 * (b->total_rows + b->count) + 16 * b->total_rows;
            break;
        case SPMV_BQ_OFFSET:
        case SPMV_BQ_N:
        case SPMV_BQ_NNZ:
        case SPMV_BQ_LANES:
            if (!mat) spmvk::fail(SPMV_EINVAL, "matrix %d", m);
            *out = what == SPMV_BQ_OFFSET ? b->mats[m].row_off
                 : what == SPMV_BQ_N      ? b->n[m]
                 : what == SPMV_BQ_NNZ    ? b->nnz[m]
                                          : b->mats[m].lanes;
            break;
        default: spmvk::fail(SPMV_EINVAL, "unknown query %d", what);
    }
    BATCH_CATCH
    return SPMV_OK;
}

int spmv_batch_run(spmv_batch* b, const double* x, double* y, cudaStream_t s) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    if (b->total_rows > 0 && (!x || !y)) spmvk::fail(SPMV_EINVAL, "x_dev or y_dev is NULL");
    if (b->n_items == 0) return SPMV_OK;
    spmvk::check_cuda(cudaMemsetAsync(b->ticket, 0, sizeof(int), s), "ticket reset");
    int grid = b->num_sms * std::max(1, b->occupancy);
    const int need = (b->n_items + kThreads / 32 - 1) / (kThreads / 32);
    if (grid > need) grid = need;
    batch_persistent_kernel<<<grid, kThreads, 0, s>>>(args_of(b, x, y));
    spmvk::check_cuda(cudaGetLastError(), "batch launch");
    BATCH_CATCH
    return SPMV_OK;
}

int spmv_batch_run_separate(spmv_batch* b, int m, const double* x, double* y, cudaStream_t s) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    if (m < -1 || m >= b->count) spmvk::fail(SPMV_EINVAL, "matrix %d", m);
    if (b->total_rows > 0 && (!x || !y)) spmvk::fail(SPMV_EINVAL, "x_dev or y_dev is NULL");
    const BatchArgs a = args_of(b, x, y);
    const int lo = m < 0 ? 0 : m, hi = m < 0 ? b->count : m + 1;
    for (int i = lo; i < hi; ++i) {
        const int first = b->item_off[i], last = b->item_off[i + 1];
        if (last <= first) continue;
        int grid = b->num_sms * std::max(1, b->occupancy);
        const int need = (last - first + kThreads / 32 - 1) / (kThreads / 32);
        if (grid > need) grid = need;
        batch_range_kernel<<<grid, kThreads, 0, s>>>(a, first, last);
        spmvk::check_cuda(cudaGetLastError(), "matrix launch");
    }
    BATCH_CATCH
    return SPMV_OK;
}

}  // extern "C"
