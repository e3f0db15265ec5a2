// Many independent CSR products in one persistent launch.
//
// The matrices of a batch live back to back in HBM (row pointers local to
// each matrix, entries padded to a multiple of 4 so every matrix starts
// 16-byte aligned).  A work item is a block of up to 256 rows of one matrix;
// persistent CTAs claim items with an atomic ticket and compute every row
// with the pair-per-lane scheme (lanes per row chosen per matrix by the
// autotuner).  The plain alternative launches the same per-row code once
// per matrix; both give bit-identical results because each row is summed
// by the same lanes in the same order.
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

// Rows [r0, r1) of one matrix: V lanes per row, lane h takes the aligned
// entry pairs h, h+V, ...; the FMA loop runs the warp's longest share.
template <int V>
__device__ __forceinline__ void batch_rows(const BatchArgs& a, const BatchMat& m, int r0, int r1,
                                           uint64_t pol) {
    constexpr int GROUPS = kThreads / V;
    constexpr int U = 4;
    const int lane = threadIdx.x % V;
    const int group = threadIdx.x / V;
    const int32_t* ptr = a.ptr + m.ptr_off;
    const int32_t* col = a.col + m.ent_off;
    const double* val = a.val + m.ent_off;
    const double* x = a.x + m.row_off;
    double* y = a.y + m.row_off;
    for (int rbase = r0; rbase < r1; rbase += GROUPS) {
        const int row = rbase + group;
        int kb = 0, ke = 0, k2 = 0, cnt = 0;
        if (row < r1) {
            kb = __ldg(ptr + row);
            ke = __ldg(ptr + row + 1);
            k2 = kb & ~1;
            const int npairs = (ke - k2 + 1) >> 1;
            cnt = npairs > lane ? (npairs - lane + V - 1) / V : 0;
        }
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
        if (row < r1 && lane == 0) y[row] = sum;
    }
}

__device__ __forceinline__ void batch_item(const BatchArgs& a, int it, uint64_t pol) {
    const BatchItem w = a.items[it];
    const BatchMat m = a.mats[w.m];
    switch (m.lanes) {
        case 1: batch_rows<1>(a, m, w.r0, w.r1, pol); break;
        case 2: batch_rows<2>(a, m, w.r0, w.r1, pol); break;
        case 4: batch_rows<4>(a, m, w.r0, w.r1, pol); break;
        case 8: batch_rows<8>(a, m, w.r0, w.r1, pol); break;
        case 16: batch_rows<16>(a, m, w.r0, w.r1, pol); break;
        default: batch_rows<32>(a, m, w.r0, w.r1, pol); break;
    }
}

// Persistent: CTAs claim items with an atomic ticket until none is left.
__global__ void __launch_bounds__(kThreads, 4) batch_persistent_kernel(BatchArgs a) {
    __shared__ int s_item;
    const uint64_t pol = policy_evict_last();
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.ticket, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= a.n_items) break;
        batch_item(a, it, pol);
    }
}

// Items [first, last) with a grid-stride loop (one matrix per launch).
__global__ void __launch_bounds__(kThreads, 4) batch_range_kernel(BatchArgs a, int first, int last) {
    const uint64_t pol = policy_evict_last();
    for (int it = first + (int)blockIdx.x; it < last; it += (int)gridDim.x) batch_item(a, it, pol);
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
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
        spmvk::fail(SPMV_EINVAL, "lanes %d not in {1,2,4,8,16,32}", lanes);
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
    if (grid > b->n_items) grid = b->n_items;
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
        if (grid > last - first) grid = last - first;
        batch_range_kernel<<<grid, kThreads, 0, s>>>(a, first, last);
        spmvk::check_cuda(cudaGetLastError(), "matrix launch");
    }
    BATCH_CATCH
    return SPMV_OK;
}

}  // extern "C"
