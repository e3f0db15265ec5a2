// Merge-path CSR product for skewed row lengths (the K-merge kernel).
//
// The rows' end offsets and the entry indices are merged into one path of
// rows + entries items (Merrill and Garland's merge-based CSR); a tile is a
// fixed run of MERGE_ITEMS items, so every CTA does the same work however
// long the rows are.  Tiles are staged in shared memory by bulk copies as
// in the thread-per-row kernel; each thread walks MERGE_IPT consecutive
// items with one DFMA per entry.  Rows cut by a thread boundary are finished
// by the thread that reaches their end, which adds the partial sums of the
// threads before it in thread order; rows cut by a tile boundary leave a
// per-tile carry that a second kernel adds in tile order.  No atomics and no
// data-dependent order: results depend only on the matrix.
#include "internal.h"
#include "pdl.cuh"

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace spmvk {

namespace {

constexpr int MERGE_NT = 256;                       // threads per CTA
constexpr int MERGE_IPT = 8;                        // items per thread
constexpr int MERGE_ITEMS = MERGE_NT * MERGE_IPT;   // items per tile
constexpr int MERGE_ST = 2;                         // stages

struct MergeLayout {
    static constexpr int VAL_N = MERGE_ITEMS + 2;
    static constexpr int COL_N = MERGE_ITEMS + 8;
    static constexpr int PTR_N = MERGE_ITEMS + 12;
    static constexpr int VAL_OFF = 0;
    static constexpr int COL_OFF = VAL_N * 8;
    static constexpr int PTR_OFF = COL_OFF + COL_N * 4;
    static constexpr int BYTES = PTR_OFF + PTR_N * 4;
    static_assert(BYTES % 16 == 0 && COL_OFF % 16 == 0 && PTR_OFF % 16 == 0, "16-byte parts");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;
constexpr uint64_t kDrainLimitNs = 100000000ull;
constexpr int kErrTimeout = 6;

}  // namespace

// Error word of launches that have no plan (CsrArgs::err == nullptr).
__device__ int g_csr_err = 0;

namespace {

__device__ __forceinline__ void put(const CsrArgs& a, int row, double v) {
    const int o = a.rowmap ? __ldg(a.rowmap + row) : row;
    a.y[o] = a.accumulate ? a.y[o] + v : v;
}

// Merge-path coordinate of diagonal d in the merge of row ends A[0..a_len)
// (A[i] = end of row i minus the entry base) with entry indices 0..b_len:
// returns the number of row ends consumed.  Row end i precedes entry j
// when A[i] <= j.
template <class F>
__device__ __forceinline__ int path_search(int d, int a_len, int b_len, F A) {
    int lo = d - b_len > 0 ? d - b_len : 0;
    int hi = d < a_len ? d : a_len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A(mid) <= d - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// GUARD: the CSR arrays are the caller's, not padded; bulk copies stop at
// the last 16-byte boundary inside each array and the few entries past it
// are read from global memory.
template <bool GUARD>
__global__ void __launch_bounds__(MERGE_NT, 3) merge_kernel(CsrArgs a, const MergeTile* __restrict__ tiles,
                                                         int tile_begin, int tile_end,
                                                         Carry* __restrict__ carries) {
    // the previous kernel of this stream is done (unless independent); the
    // next kernel is this operation's fixup, which needs the carries
    pdl_begin(a.pdl & kPdlNoWait);
    using L = MergeLayout;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[MERGE_ST];
    __shared__ int c_row[MERGE_NT];
    __shared__ double c_val[MERGE_NT];
    __shared__ int w_key[MERGE_NT / 32];
    __shared__ double w_val[MERGE_NT / 32];
    __shared__ int w_start[MERGE_NT / 32];

    const int tid = threadIdx.x;
    const int first = tile_begin + (int)blockIdx.x;
    const int stride = (int)gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < MERGE_ST; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // staged ranges of one tile: values [va, vb), columns [ca, cb), row
    // pointers [pa, pb) covering ptr[r0 .. r1]
    struct Span { int va, vb, ca, cb, pa, pb; };
    auto span_of = [&](const MergeTile& d) {
        Span x;
        x.va = d.k0 & ~1;
        x.vb = (d.k1 + 1) & ~1;
        x.ca = d.k0 & ~3;
        x.cb = (d.k1 + 3) & ~3;
        x.pa = d.r0 & ~3;
        x.pb = (d.r1 + 4) & ~3;
        if (GUARD) {
            const int ve = a.nnz_total & ~1, ce = a.nnz_total & ~3, pe = (a.n_rows + 1) & ~3;
            x.vb = x.vb < ve ? x.vb : ve;
            x.cb = x.cb < ce ? x.cb : ce;
            x.pb = x.pb < pe ? x.pb : pe;
            if (x.vb < x.va) x.vb = x.va;
            if (x.cb < x.ca) x.cb = x.ca;
            if (x.pb < x.pa) x.pb = x.pa;
        }
        return x;
    };

    auto issue = [&](int j) {
        const int t = first + j * stride;
        if (t >= tile_end) return;
        const int s = j % MERGE_ST;
        const MergeTile d = tiles[t];
        const uint32_t bar = smem_u32(&bars[s]);
        const Span x = span_of(d);
        const uint32_t vbytes = (uint32_t)(x.vb - x.va) * 8u;
        const uint32_t cbytes = (uint32_t)(x.cb - x.ca) * 4u;
        const uint32_t pbytes = (uint32_t)(x.pb - x.pa) * 4u;
        const int va = x.va, ca = x.ca, pa = x.pa;
        unsigned char* st = smem + (size_t)s * L::BYTES;
        mbar_arrive_expect_tx(bar, vbytes + cbytes + pbytes);
        if (vbytes) bulk_g2s(smem_u32(st + L::VAL_OFF), a.val + va, vbytes, bar);
        if (cbytes) bulk_g2s(smem_u32(st + L::COL_OFF), a.col + ca, cbytes, bar);
        if (pbytes) bulk_g2s(smem_u32(st + L::PTR_OFF), a.ptr + pa, pbytes, bar);
    };

    if (tid == 0)
        for (int j = 0; j < MERGE_ST - 1; ++j) issue(j);

    int j = 0;
    bool aborted = false;
    for (;; ++j) {
        const int t = first + j * stride;
        if (t >= tile_end) break;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(j + MERGE_ST - 1);
        }
        const int s = j % MERGE_ST;
        bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((j / MERGE_ST) & 1), kWaitLimitNs);
        if (a.abort_tile > 0 && t >= a.abort_tile - 1) ok = false;   // test hook: the stage has landed
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        const MergeTile d = tiles[t];
        const unsigned char* st = smem + (size_t)s * L::BYTES;
        const double* vs = reinterpret_cast<const double*>(st + L::VAL_OFF);
        const int32_t* cs = reinterpret_cast<const int32_t*>(st + L::COL_OFF);
        const int32_t* ps = reinterpret_cast<const int32_t*>(st + L::PTR_OFF);
        const Span x = span_of(d);
        auto ptr_at = [&](int r) { return (!GUARD || r < x.pb) ? ps[r - x.pa] : __ldg(a.ptr + r); };
        auto val_at = [&](int kg) { return (!GUARD || kg < x.vb) ? vs[kg - x.va] : __ldg(a.val + kg); };
        auto col_at = [&](int kg) { return (!GUARD || kg < x.cb) ? cs[kg - x.ca] : __ldg(a.col + kg); };
        // end of row r0 + i relative to the tile's first entry (i < a_len)
        auto row_end_rel = [&](int i) { return ptr_at(d.r0 + i + 1) - d.k0; };
        const int a_len = d.r1 - d.r0, b_len = d.k1 - d.k0;
        const int items = a_len + b_len;
        const int d0 = tid * MERGE_IPT < items ? tid * MERGE_IPT : items;
        const int d1 = d0 + MERGE_IPT < items ? d0 + MERGE_IPT : items;
        int i = path_search(d0, a_len, b_len, row_end_rel);
        int k = d0 - i;   // entries consumed, relative to k0
        // the thread's range ends at (i_end, k_end); its entries are
        // k .. k_end-1 (at most MERGE_IPT), gathered up front so the
        // loads are in flight together
        const int i_end = path_search(d1, a_len, b_len, row_end_rel);
        const int k_end = d1 - i_end;
        // does this thread start inside a row whose earlier entries belong to
        // a previous thread or tile?
        bool open_head = (k + d.k0) > ptr_at(d.r0 + i);
        bool partial = false;
        int head_row = -1;
        double head_val = 0.0;
        double sum = 0.0;
        const double* xb = a.x + d.xoff;
        double vv[MERGE_IPT], xv[MERGE_IPT];
#pragma unroll
        for (int u = 0; u < MERGE_IPT; ++u) {
            const bool m = k + u < k_end;
            const int kg = k + u + d.k0;
            vv[u] = m ? val_at(kg) : 0.0;
            xv[u] = __ldg(xb + (m ? col_at(kg) : 0));
        }
        // walk the merge path: row end i comes before entry j when
        // row_end(i) <= j; rows i < i_end end inside this range
        auto close_row = [&]() {
            if (open_head) {
                head_row = i;
                head_val = sum;
                open_head = false;
            } else {
                put(a, d.r0 + i, sum);
            }
            sum = 0.0;
            partial = false;
            ++i;
        };
#pragma unroll
        for (int u = 0; u < MERGE_IPT; ++u) {
            if (k + u < k_end) {
                while (i < i_end && row_end_rel(i) <= k + u) close_row();
                sum = fma(vv[u], xv[u], sum);
                partial = true;
            }
        }
        while (i < i_end) close_row();
        k = k_end;
        // Rows cut between threads: S[t] = the partial sums of the run of
        // threads ending at t that carry t's open row, combined by a
        // segmented scan in a fixed tree order (shuffles within a warp, then
        // the earlier warps of the run), so the result is deterministic.
        const int key = partial ? i : -1;   // row still open after t's items
        c_row[tid] = key;
        __syncthreads();
        const int lane = tid & 31, warp = tid >> 5;
        double v = key >= 0 ? sum : 0.0;
        int f = (key < 0 || tid == 0 || c_row[tid - 1] != key) ? 1 : 0;   // run starts here
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double vu = __shfl_up_sync(0xffffffffu, v, off);
            const int fu = __shfl_up_sync(0xffffffffu, f, off);
            if (lane >= off) {
                if (!f) v = vu + v;
                f |= fu;
            }
        }
        if (lane == 31) {
            w_key[warp] = key;
            w_val[warp] = v;
            w_start[warp] = f;
        }
        __syncthreads();
        if (!f) {   // the run began in an earlier warp
            double cin = 0.0;
            for (int w = warp - 1; w >= 0 && w_key[w] == key; --w) {
                cin = w_val[w] + cin;
                if (w_start[w]) break;
            }
            v = cin + v;
        }
        c_val[tid] = v;
        __syncthreads();
        // a row this thread finished after earlier threads started it
        if (head_row >= 0) {
            const double tot = (tid > 0 && c_row[tid - 1] == head_row) ? c_val[tid - 1] + head_val
                                                                       : head_val;
            put(a, d.r0 + head_row, tot);
        }
        // the tile's carry: the row still open after the tile's last item
        const int last = (items + MERGE_IPT - 1) / MERGE_IPT - 1;
        if (tid == (last >= 0 ? last : 0)) {
            Carry c{-1, 0, 0.0};
            if (last >= 0 && c_row[last] >= 0) {
                c.row = d.r0 + c_row[last];
                c.val = c_val[last];
            }
            carries[t] = c;
        }
        __syncthreads();
    }
    if (aborted && tid == 0) {
        atomicExch(a.err ? a.err : &g_csr_err, kErrTimeout);
        // the tiles this CTA will not finish carry nothing, so the fixup
        // kernel never reads a carry left by an earlier launch
        for (int jj = j; first + jj * stride < tile_end; ++jj) carries[first + jj * stride] = Carry{-1, 0, 0.0};
        for (int jj = j + 1; jj < j + MERGE_ST; ++jj) {
            if (first + jj * stride >= tile_end) break;
            mbar_wait_bounded(smem_u32(&bars[jj % MERGE_ST]), (uint32_t)((jj / MERGE_ST) & 1), kDrainLimitNs);
        }
    }
}

// Adds tile carries to their rows: the first tile of each run of tiles
// carrying the same row sums the run in tile order and adds it once.
__global__ void __launch_bounds__(256) merge_fixup_kernel(CsrArgs a, const Carry* __restrict__ carries,
                                                          int tile_begin, int tile_end) {
    pdl_begin(a.pdl & kPdlEarly);   // the carries of the merge kernel are complete
    const int t = tile_begin + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= tile_end) return;
    const Carry c = carries[t];
    if (c.row < 0 || c.row >= a.n_rows) return;   // none, or not a row of this product
    if (t > tile_begin && carries[t - 1].row == c.row) return;
    double tot = c.val;
    for (int u = t + 1; u < tile_end && carries[u].row == c.row; ++u) tot += carries[u].val;
    const int o = a.rowmap ? __ldg(a.rowmap + c.row) : c.row;
    a.y[o] += tot;
}

// Merge-path coordinates of every tile boundary, computed on the device
// from a CSR row pointer: tile t covers diagonals [t*ITEMS, (t+1)*ITEMS).
__global__ void merge_partition_kernel(const int32_t* __restrict__ ptr, int row_begin, int row_end,
                                       int32_t xoff, MergeTile* __restrict__ tiles, int n_tiles) {
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= n_tiles) return;
    const int k_base = __ldg(ptr + row_begin);
    const int a_len = row_end - row_begin;
    const int b_len = __ldg(ptr + row_end) - k_base;
    const int items = a_len + b_len;
    auto A = [&](int i) { return __ldg(ptr + row_begin + i + 1) - k_base; };
    const int d0 = t * MERGE_ITEMS;
    const int d1 = d0 + MERGE_ITEMS < items ? d0 + MERGE_ITEMS : items;
    const int i0 = path_search(d0, a_len, b_len, A);
    const int i1 = path_search(d1, a_len, b_len, A);
    MergeTile m{};
    m.r0 = row_begin + i0;
    m.r1 = row_begin + i1;
    m.k0 = k_base + d0 - i0;
    m.k1 = k_base + d1 - i1;
    m.xoff = xoff;
    tiles[t] = m;
}

}  // namespace

int merge_items_per_tile() { return MERGE_ITEMS; }

template <bool GUARD>
static cudaError_t run_merge(const CsrArgs& a, const MergeTile* tiles, int tile_begin, int tile_end,
                             Carry* carries, int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)MERGE_ST * MergeLayout::BYTES;
    static std::atomic<unsigned long long> configured{0};   // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(configured.load(std::memory_order_acquire) >> dev & 1ull)) {
        e = cudaFuncSetAttribute(merge_kernel<GUARD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured.fetch_or(1ull << dev, std::memory_order_acq_rel);
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, merge_kernel<GUARD>, MERGE_NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int grid = num_sms * occ;
    if (grid > tile_end - tile_begin) grid = tile_end - tile_begin;
    return launch_pdl(merge_kernel<GUARD>, dim3(grid), dim3(MERGE_NT), smem, s, a, tiles, tile_begin, tile_end,
                      carries);
}

cudaError_t launch_merge(const CsrArgs& a, const MergeTile* tiles, int tile_begin, int tile_end,
                         Carry* carries, int num_sms, cudaStream_t s) {
    if (tile_end <= tile_begin) return cudaSuccess;
    cudaError_t e = a.guarded ? run_merge<true>(a, tiles, tile_begin, tile_end, carries, num_sms, s)
                              : run_merge<false>(a, tiles, tile_begin, tile_end, carries, num_sms, s);
    if (e != cudaSuccess) return e;
    const int n = tile_end - tile_begin;
    return launch_pdl(merge_fixup_kernel, dim3((n + 255) / 256), dim3(256), 0, s, a, carries, tile_begin, tile_end);
}

cudaError_t launch_merge_partition(const int32_t* ptr, int row_begin, int row_end, int32_t xoff,
                                   MergeTile* tiles, int n_tiles, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    merge_partition_kernel<<<(n_tiles + 127) / 128, 128, 0, s>>>(ptr, row_begin, row_end, xoff, tiles,
                                                                 n_tiles);
    return cudaGetLastError();
}

cudaError_t read_clear_csr_error(int* out) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_csr_err, sizeof(int));
    if (e != cudaSuccess) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_csr_err, &zero, sizeof(int));
}

// ------------------------------------------------------------------------
// Fixed scratch for the no-allocation entry point.  Every GPU that loads the
// library holds this array until the process exits.  Its name is only a
// host-side stand-in in host code: the device address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
// ------------------------------------------------------------------------
constexpr int kNoAllocMaxTiles = 65536;
constexpr size_t kNoAllocTileBytes = (size_t)kNoAllocMaxTiles * sizeof(MergeTile);
constexpr size_t kNoAllocBytes = kNoAllocTileBytes + (size_t)kNoAllocMaxTiles * sizeof(Carry);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

int64_t noalloc_max_items() { return (int64_t)kNoAllocMaxTiles * MERGE_ITEMS; }

cudaError_t launch_merge_noalloc(const CsrArgs& a, int num_sms, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_noalloc_addr[dev] = base;
        }
        base = g_noalloc_addr[dev];
    }
    const int64_t items = (int64_t)a.n_rows + a.nnz_total;
    if (items > noalloc_max_items()) return cudaErrorInvalidValue;
    const int n_tiles = (int)((items + MERGE_ITEMS - 1) / MERGE_ITEMS);
    MergeTile* tiles = static_cast<MergeTile*>(base);
    Carry* carries = reinterpret_cast<Carry*>(static_cast<unsigned char*>(base) + kNoAllocTileBytes);
    // tiles [0, n_tiles) and their carries are rewritten before they are
    // read, so nothing left by an earlier call is ever used
    e = launch_merge_partition(a.ptr, 0, a.n_rows, 0, tiles, n_tiles, s);
    if (e != cudaSuccess) return e;
    return launch_merge(a, tiles, 0, n_tiles, carries, num_sms, s);
}

}  // namespace spmvk
