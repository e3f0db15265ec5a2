// Kernels of the row-partitioned FP64 SpMV (Sec. III-A, Fig. 3 of Pearson,
// Javeed and Devine): the Pack gather, the halo exchange copy, and the CSR
// products y_L = A_L x_L and y += A_R x_R.
//
// Design for sm_103a: FP64 FMA issues at 2 lanes/clk/SM on this part, so a
// CSR product with HBM at full speed is nearly FP64-bound.  Every product
// kernel therefore spends exactly one DFMA per stored entry on the main path
// (one thread walks a row), and gets coalescing from bulk copies
// (cp.async.bulk, the TMA engine) of whole tiles into a shared-memory ring
// instead of from lanes cooperating on a row, which would cost FP64 adds in
// shuffle reductions.  Every row is summed by one thread in storage order,
// so results do not depend on the grid, the stream or the schedule.
#include "internal.h"
#include "pdl.cuh"

#include <cuda_runtime.h>

#include <atomic>

namespace spmvk {

// ------------------------------------------------------------------------
// PTX helpers: mbarrier, bulk copy, global timer
// ------------------------------------------------------------------------
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
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx)
                 : "memory");
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
// Wait for phase `parity` of an mbarrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}
// Bulk copy global -> shared (16-byte aligned addresses, size % 16 == 0),
// completion reported to an mbarrier as transaction bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// Bulk copy with an L2 eviction policy (evict-first for data read once).
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Read-only load of x kept in L2 (x is gathered many times per product).
__device__ __forceinline__ double ldg_keep(const double* p, uint64_t policy) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(policy));
    return v;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // 1 s per wait
constexpr uint64_t kDrainLimitNs = 100000000ull;   // 0.1 s per drain wait
constexpr int kErrTimeout = 6;                     // -SPMV_ETIMEOUT

__device__ __forceinline__ void store_row(const CsrArgs& a, int row, double sum) {
    if (a.rowmap) {
        const int o = __ldg(a.rowmap + row);
        a.y[o] = a.accumulate ? a.y[o] + sum : sum;
    } else {
        a.y[row] = a.accumulate ? a.y[row] + sum : sum;
    }
}

// ------------------------------------------------------------------------
// Pack: dst[k] = x[idx[k]] for every slot k (pos == nullptr) or for the
// slots listed in pos[0..count).  A thread takes kPackIlp slots a grid
// stride apart per step: their index loads, then their gathers, then their
// stores, so kPackIlp index-then-gather chains are in flight at once.
// ------------------------------------------------------------------------
constexpr int kPackIlp = 4;

__global__ void __launch_bounds__(256) gather_kernel(const double* __restrict__ x,
                                                     const int32_t* __restrict__ idx,
                                                     const int32_t* __restrict__ pos,
                                                     double* __restrict__ dst, int64_t count, int pdl) {
    pdl_begin(pdl);  // the previous kernel of this stream is done (unless independent)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < count; i0 += kPackIlp * stride) {
        int64_t k[kPackIlp];
        int32_t c[kPackIlp];
        double v[kPackIlp];
#pragma unroll
        for (int u = 0; u < kPackIlp; ++u) {
            const int64_t i = i0 + u * stride;
            k[u] = i < count ? (pos ? (int64_t)__ldg(pos + i) : i) : -1;
        }
#pragma unroll
        for (int u = 0; u < kPackIlp; ++u) c[u] = k[u] >= 0 ? __ldg(idx + k[u]) : 0;
#pragma unroll
        for (int u = 0; u < kPackIlp; ++u) v[u] = k[u] >= 0 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < kPackIlp; ++u)
            if (k[u] >= 0) dst[k[u]] = v[u];
    }
}

cudaError_t launch_gather(const double* x, const int32_t* idx, const int32_t* pos,
                          double* dst, int64_t count, int num_sms, cudaStream_t s, int pdl) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 256 * kPackIlp - 1) / (256 * kPackIlp);
    const int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    return launch_pdl(gather_kernel, dim3((unsigned)blocks), dim3(256), 0, s, x, idx, pos, dst, count, pdl);
}

// ------------------------------------------------------------------------
// Halo exchange: dst[0..count) = src[0..count).  Aligned: 16-byte pairs,
// kPackIlp loads in flight per thread before their stores.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) copy_kernel(const double* __restrict__ src,
                                                   double* __restrict__ dst, int64_t count, int pdl) {
    pdl_begin(pdl);  // the previous kernel of this stream is done (unless independent)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    if (vec) {
        const int64_t pairs = count >> 1;
        const double2* s2 = reinterpret_cast<const double2*>(src);
        double2* d2 = reinterpret_cast<double2*>(dst);
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < pairs; i0 += kPackIlp * stride) {
            double2 t[kPackIlp];
#pragma unroll
            for (int u = 0; u < kPackIlp; ++u)
                if (i0 + u * stride < pairs) t[u] = __ldg(s2 + i0 + u * stride);
#pragma unroll
            for (int u = 0; u < kPackIlp; ++u)
                if (i0 + u * stride < pairs) d2[i0 + u * stride] = t[u];
        }
        if ((count & 1) && blockIdx.x == 0 && threadIdx.x == 0) dst[count - 1] = src[count - 1];
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
            dst[i] = __ldg(src + i);
    }
}

cudaError_t launch_copy(const double* src, double* dst, int64_t count, int num_sms,
                        cudaStream_t s, int pdl) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count / 2 + 256 * kPackIlp - 1) / (256 * kPackIlp);
    if (blocks < 1) blocks = 1;
    // 8 CTAs per SM: a 13 MB halo (a power-law rank's) in one round of loads
    // (3.8 us per rank against 4.2 us at 4 CTAs per SM; the 104 MB exchange
    // 32.5 us, 0.94 of the copy peak)
    const int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    return launch_pdl(copy_kernel, dim3((unsigned)blocks), dim3(256), 0, s, src, dst, count, pdl);
}

// ------------------------------------------------------------------------
// Thread-per-row CSR product over bulk-copied tiles.
//
// Persistent CTAs walk tiles tile_begin + blockIdx.x + j * gridDim.x.  One
// elected thread copies each tile's values, columns and row pointers into a
// ring of ST shared-memory stages with cp.async.bulk (start addresses rounded
// down to 16 bytes, sizes rounded up; the device arrays are padded so the
// rounded reads stay in bounds).  Thread i of the CTA sums row r0 + i of the
// tile in storage order with one DFMA per entry.
// ------------------------------------------------------------------------
template <int ROWS, int CAP>
struct TileLayout {
    static constexpr int VAL_N = CAP + 2;    // doubles: k0 rounded down to even, k1 up
    static constexpr int COL_N = CAP + 8;    // ints: rounded to multiples of 4
    static constexpr int PTR_N = ROWS + 8;   // ints: rows r0..r1 inclusive, rounded
    static constexpr int VAL_OFF = 0;
    static constexpr int COL_OFF = VAL_N * 8;
    static constexpr int PTR_OFF = COL_OFF + COL_N * 4;
    static constexpr int BYTES = PTR_OFF + PTR_N * 4;
    static_assert(CAP % 4 == 0 && ROWS % 4 == 0, "16-byte aligned stage parts");
    static_assert(BYTES % 16 == 0, "stage size keeps 16-byte alignment");
};

template <int NT, int CAP, int ST, int CH, int LANES>
__global__ void __launch_bounds__(NT, 1) csr_tile_kernel(CsrArgs a, const Tile* __restrict__ tiles,
                                                      int tile_begin, int tile_end) {
    pdl_begin(a.pdl);  // the previous kernel of this stream is done (unless independent)
    static_assert(LANES == 1 || LANES == 2 || LANES == 4, "lanes per row");
    using L = TileLayout<NT / LANES, CAP>;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[ST];
    __shared__ double red[NT];

    const int tid = threadIdx.x;
    const int first = tile_begin + (int)blockIdx.x;
    const int stride = (int)gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < ST; ++s) mbar_init(smem_u32(&bars[s]), 1);
        mbar_fence_init();
    }
    __syncthreads();

    // Producer: thread 0 issues the copies of the j-th tile of this CTA.
    auto issue = [&](int j) {
        const int t = first + j * stride;
        if (t >= tile_end) return;
        const int s = j % ST;
        const Tile d = tiles[t];
        const uint32_t bar = smem_u32(&bars[s]);
        if (d.flags & TILE_LONG) {
            mbar_arrive_expect_tx(bar, 0);
            return;
        }
        const int va = d.k0 & ~1, vb = (d.k1 + 1) & ~1;
        const int ca = d.k0 & ~3, cb = (d.k1 + 3) & ~3;
        const int pa = d.r0 & ~3, pb = (d.r1 + 4) & ~3;
        const uint32_t vbytes = (uint32_t)(vb - va) * 8u;
        const uint32_t cbytes = (uint32_t)(cb - ca) * 4u;
        const uint32_t pbytes = (uint32_t)(pb - pa) * 4u;
        unsigned char* st = smem + (size_t)s * L::BYTES;
        mbar_arrive_expect_tx(bar, vbytes + cbytes + pbytes);
        if (vbytes) bulk_g2s_hint(smem_u32(st + L::VAL_OFF), a.val + va, vbytes, bar, pol_stream);
        if (cbytes) bulk_g2s_hint(smem_u32(st + L::COL_OFF), a.col + ca, cbytes, bar, pol_stream);
        bulk_g2s_hint(smem_u32(st + L::PTR_OFF), a.ptr + pa, pbytes, bar, pol_stream);
    };

    if (tid == 0) {
        for (int j = 0; j < ST - 1; ++j) issue(j);
    }

    int j = 0;
    bool aborted = false;
    for (;; ++j) {
        const int t = first + j * stride;
        if (t >= tile_end) break;
        if (tid == 0) {
            // stage (j-1) % ST was released by the barrier that ended j-1
            fence_proxy_async_smem();
            issue(j + ST - 1);
        }
        const int s = j % ST;
        const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((j / ST) & 1), kWaitLimitNs);
        // every thread leaves together if any wait gave up
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        const Tile d = tiles[t];
        {
            if (d.flags & TILE_LONG) {
                // one row longer than a stage: the CTA sums it from global
                // memory with a fixed-order tree, so the result is still
                // independent of the launch.
                const double* xb = a.x + d.xoff;
                double part = 0.0;
                for (int k = d.k0 + tid; k < d.k1; k += NT)
                    part = fma(__ldg(a.val + k), __ldg(xb + __ldg(a.col + k)), part);
                red[tid] = part;
                __syncthreads();
                for (int w = NT / 2; w > 0; w >>= 1) {
                    if (tid < w) red[tid] += red[tid + w];
                    __syncthreads();
                }
                if (tid == 0) store_row(a, d.r0, red[0]);
            } else {
                // LANES threads share a row: thread h takes entries
                // kb + h, kb + h + LANES, ...; the FMA loop runs as many
                // times as the warp's longest share, and the LANES partial
                // sums meet in a fixed xor-butterfly
                const int row = d.r0 + tid / LANES;
                const int h = tid % LANES;
                const unsigned char* st = smem + (size_t)s * L::BYTES;
                const double* vs = reinterpret_cast<const double*>(st + L::VAL_OFF);
                const int32_t* cs = reinterpret_cast<const int32_t*>(st + L::COL_OFF);
                const int32_t* ps = reinterpret_cast<const int32_t*>(st + L::PTR_OFF);
                const int va = d.k0 & ~1, ca = d.k0 & ~3, pa = d.r0 & ~3;
                const int dc = va - ca;   // column slot of value slot 0
                int kb = 0, cnt = 0;
                if (row < d.r1) {
                    kb = ps[row - pa] - va + h;
                    const int ke = ps[row + 1 - pa] - va;
                    cnt = ke > kb ? (ke - kb + LANES - 1) / LANES : 0;
                }
                const int wmax = __reduce_max_sync(0xffffffffu, cnt);
                const double* xb = a.x + d.xoff;
                double sum = 0.0;
                for (int base = 0; base < wmax; base += CH) {
                    // CH gathers in flight before their FMAs; slots past
                    // the share read x[xoff] (a valid address) so every
                    // load is unconditional, and their FMA results are
                    // discarded; FMAs still run in storage order
                    double xv[CH], vv[CH];
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        const bool m = base + u < cnt;
                        const int k = kb + LANES * (base + u);
                        const int c = m ? cs[k + dc] : 0;
                        vv[u] = m ? vs[k] : 0.0;
                        xv[u] = ldg_keep(xb + c, pol_keep);
                    }
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        if (base + u >= wmax) break;   // warp-uniform
                        const double t = fma(vv[u], xv[u], sum);
                        sum = (base + u < cnt) ? t : sum;
                    }
                }
#pragma unroll
                for (int off = LANES / 2; off > 0; off >>= 1)
                    sum += __shfl_xor_sync(0xffffffffu, sum, off, LANES);
                if (row < d.r1 && h == 0) store_row(a, row, sum);
            }
        }
        __syncthreads();   // stage s is free again
    }
    if (aborted && tid == 0) {
        atomicExch(a.err, kErrTimeout);
        // let the copies still in flight land before the CTA leaves
        for (int jj = j + 1; jj < j + ST; ++jj) {
            if (first + jj * stride >= tile_end) break;
            mbar_wait_bounded(smem_u32(&bars[jj % ST]), (uint32_t)((jj / ST) & 1), kDrainLimitNs);
        }
    }
}

template <int NT, int CAP, int ST, int CH, int LANES>
static cudaError_t run_tile(const CsrArgs& a, const Tile* tiles, int tb, int te, int num_sms,
                            cudaStream_t s) {
    using L = TileLayout<NT / LANES, CAP>;
    const size_t smem = (size_t)ST * L::BYTES;
    static std::atomic<unsigned long long> configured{0};   // one bit per device ordinal
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev >= 64 || !(configured.load(std::memory_order_acquire) >> dev & 1ull)) {
        cudaError_t e = cudaFuncSetAttribute(csr_tile_kernel<NT, CAP, ST, CH, LANES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured.fetch_or(1ull << dev, std::memory_order_acq_rel);
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, csr_tile_kernel<NT, CAP, ST, CH, LANES>,
                                                                  NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int n_tiles = te - tb;
    int grid = num_sms * occ;
    if (grid > n_tiles) grid = n_tiles;
    return launch_pdl(csr_tile_kernel<NT, CAP, ST, CH, LANES>, dim3(grid), dim3(NT), smem, s, a, tiles, tb, te);
}

template <int NT, int CAP, int ST, int CH, int LANES>
static int ctas_per_sm_of() {
    using L = TileLayout<NT / LANES, CAP>;
    const size_t smem = (size_t)ST * L::BYTES;
    cudaFuncSetAttribute(csr_tile_kernel<NT, CAP, ST, CH, LANES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, csr_tile_kernel<NT, CAP, ST, CH, LANES>, NT, smem) !=
        cudaSuccess)
        return 0;
    return occ;
}

// The geometries compiled into the library (threads, entries per stage,
// stages).  The plan builds its tiles for one of them.
// (threads, entries per stage, stages, gathers per chunk, threads per row)
#define SPMV_TILE_GEOMS(X)      \
    X(256, 3456, 2, 16, 2)      \
    X(512, 6912, 2, 16, 2)      \
    X(256, 3456, 3, 16, 2)      \
    X(128, 3456, 2, 32, 1)      \
    X(256, 2048, 3, 8, 2)

TileGeom default_tile_geom() { return TileGeom{256, 3456, 2, 16, 2}; }

#define GEOM_IS(nt, cap, st, ch, ln) \
    (g.threads == nt && g.nnz_cap == cap && g.stages == st && g.chunk == ch && g.lanes == ln)

bool tile_geom_supported(const TileGeom& g) {
#define X(nt, cap, st, ch, ln) \
    if (GEOM_IS(nt, cap, st, ch, ln)) return true;
    SPMV_TILE_GEOMS(X)
#undef X
    return false;
}

int tile_ctas_per_sm(const TileGeom& g) {
#define X(nt, cap, st, ch, ln) \
    if (GEOM_IS(nt, cap, st, ch, ln)) return ctas_per_sm_of<nt, cap, st, ch, ln>();
    SPMV_TILE_GEOMS(X)
#undef X
    return 0;
}

cudaError_t launch_tile(const CsrArgs& a, const Tile* tiles, int tile_begin, int tile_end,
                        const TileGeom& g, int num_sms, cudaStream_t s) {
    if (tile_end <= tile_begin) return cudaSuccess;
#define X(nt, cap, st, ch, ln) \
    if (GEOM_IS(nt, cap, st, ch, ln)) \
        return run_tile<nt, cap, st, ch, ln>(a, tiles, tile_begin, tile_end, num_sms, s);
    SPMV_TILE_GEOMS(X)
#undef X
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------
// Vector-per-row CSR: V lanes share a row; each lane reads 4 consecutive
// entries per step with 128-bit loads (two double2 values, one int4 of
// columns) from a 4-aligned start, masks entries outside the row, and the
// V partial sums meet in a fixed xor-butterfly.  Rows come from the same
// tile table (rows r0..r1 with their x offset).
// ------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(256) csr_vector_kernel(CsrArgs a, const Tile* __restrict__ tiles,
                                                         int tile_begin, int tile_end) {
    pdl_begin(a.pdl);  // the previous kernel of this stream is done (unless independent)
    constexpr int GROUPS = 256 / V;
    const uint64_t pol_keep = policy_evict_last();
    const int lane = threadIdx.x % V;
    const int group = threadIdx.x / V;
    for (int t = tile_begin + (int)blockIdx.x; t < tile_end; t += (int)gridDim.x) {
        const Tile d = tiles[t];
        const double* xb = a.x + d.xoff;
        for (int rbase = d.r0; rbase < d.r1; rbase += GROUPS) {
            const int row = rbase + group;
            double sum = 0.0;
            if (row < d.r1) {
                const int kb = __ldg(a.ptr + row), ke = __ldg(a.ptr + row + 1);
                for (int k4 = (kb & ~3) + 4 * lane; k4 < ke; k4 += 4 * V) {
                    const int4 c = __ldg(reinterpret_cast<const int4*>(a.col + k4));
                    const double2 v0 = __ldg(reinterpret_cast<const double2*>(a.val + k4));
                    const double2 v1 = __ldg(reinterpret_cast<const double2*>(a.val + k4 + 2));
                    const bool m0 = k4 + 0 >= kb && k4 + 0 < ke, m1 = k4 + 1 >= kb && k4 + 1 < ke;
                    const bool m2 = k4 + 2 >= kb && k4 + 2 < ke, m3 = k4 + 3 >= kb && k4 + 3 < ke;
                    // masked slots read x[xoff]: entries of a neighbouring
                    // row may index another rank's block
                    const double x0 = ldg_keep(xb + (m0 ? c.x : 0), pol_keep);
                    const double x1 = ldg_keep(xb + (m1 ? c.y : 0), pol_keep);
                    const double x2 = ldg_keep(xb + (m2 ? c.z : 0), pol_keep);
                    const double x3 = ldg_keep(xb + (m3 ? c.w : 0), pol_keep);
                    double t;
                    t = fma(v0.x, x0, sum); sum = m0 ? t : sum;
                    t = fma(v0.y, x1, sum); sum = m1 ? t : sum;
                    t = fma(v1.x, x2, sum); sum = m2 ? t : sum;
                    t = fma(v1.y, x3, sum); sum = m3 ? t : sum;
                }
            }
#pragma unroll
            for (int off = V / 2; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off, V);
            if (row < d.r1 && lane == 0) store_row(a, row, sum);
        }
    }
}

// ------------------------------------------------------------------------
// Warp-private pipelines: every warp owns an ST-stage ring of 32-row tiles
// (values, columns, row pointers) in shared memory, filled by bulk copies its
// lane 0 issues against the warp's own mbarriers.  There is no block-wide
// barrier after set-up, so warps never wait for each other.  One thread per
// row, exactly one DFMA per entry in storage order (the FMA loop runs the
// warp's longest row), CH gathers of x in flight per chunk.  A row longer
// than a stage (TILE_LONG) is summed by the 32 lanes from global memory with
// a fixed butterfly.
// ------------------------------------------------------------------------
template <int WARPS, int CAP, int ST, int CH>
__global__ void __launch_bounds__(WARPS * 32, 1) csr_warp_kernel(CsrArgs a, const Tile* __restrict__ tiles,
                                                                int tile_begin, int tile_end) {
    pdl_begin(a.pdl);  // the previous kernel of this stream is done (unless independent)
    using L = TileLayout<32, CAP>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[WARPS][ST];
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    unsigned char* ring = smem + (size_t)w * ST * L::BYTES;
    const int first = tile_begin + (int)blockIdx.x * WARPS + w;
    const int stride = (int)gridDim.x * WARPS;
    if (lane == 0) {
        for (int s = 0; s < ST; ++s) mbar_init(smem_u32(&bars[w][s]), 1);
        mbar_fence_init();
    }
    __syncwarp();

    auto issue = [&](int j) {   // lane 0 only
        const int t = first + j * stride;
        if (t >= tile_end) return;
        const int s = j % ST;
        const Tile d = tiles[t];
        const uint32_t bar = smem_u32(&bars[w][s]);
        if (d.flags & TILE_LONG) {
            mbar_arrive_expect_tx(bar, 0);
            return;
        }
        const int va = d.k0 & ~1, vb = (d.k1 + 1) & ~1;
        const int ca = d.k0 & ~3, cb = (d.k1 + 3) & ~3;
        const int pa = d.r0 & ~3, pb = (d.r1 + 4) & ~3;
        const uint32_t vbytes = (uint32_t)(vb - va) * 8u;
        const uint32_t cbytes = (uint32_t)(cb - ca) * 4u;
        const uint32_t pbytes = (uint32_t)(pb - pa) * 4u;
        unsigned char* st = ring + (size_t)s * L::BYTES;
        mbar_arrive_expect_tx(bar, vbytes + cbytes + pbytes);
        if (vbytes) bulk_g2s_hint(smem_u32(st + L::VAL_OFF), a.val + va, vbytes, bar, pol_stream);
        if (cbytes) bulk_g2s_hint(smem_u32(st + L::COL_OFF), a.col + ca, cbytes, bar, pol_stream);
        bulk_g2s_hint(smem_u32(st + L::PTR_OFF), a.ptr + pa, pbytes, bar, pol_stream);
    };

    if (lane == 0)
        for (int j = 0; j < ST - 1; ++j) issue(j);
    int j = 0;
    bool aborted = false;
    for (;; ++j) {
        const int t = first + j * stride;
        if (t >= tile_end) break;
        if (lane == 0) {
            fence_proxy_async_smem();   // stage (j-1) % ST was released by the warp
            issue(j + ST - 1);
        }
        const int s = j % ST;
        const bool ok = mbar_wait_bounded(smem_u32(&bars[w][s]), (uint32_t)((j / ST) & 1), kWaitLimitNs);
        if (__any_sync(0xffffffffu, !ok)) {
            aborted = true;
            break;
        }
        const Tile d = tiles[t];
        const double* xb = a.x + d.xoff;
        if (d.flags & TILE_LONG) {
            double part = 0.0;
            for (int k = d.k0 + lane; k < d.k1; k += 32)
                part = fma(__ldg(a.val + k), ldg_keep(xb + __ldg(a.col + k), pol_keep), part);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) store_row(a, d.r0, part);
        } else {
            const unsigned char* st = ring + (size_t)s * L::BYTES;
            const double* vs = reinterpret_cast<const double*>(st + L::VAL_OFF);
            const int32_t* cs = reinterpret_cast<const int32_t*>(st + L::COL_OFF);
            const int32_t* ps = reinterpret_cast<const int32_t*>(st + L::PTR_OFF);
            const int va = d.k0 & ~1, ca = d.k0 & ~3, pa = d.r0 & ~3;
            const int dc = va - ca;
            const int row = d.r0 + lane;
            int kb = 0, cnt = 0;
            if (row < d.r1) {
                kb = ps[row - pa] - va;
                cnt = ps[row + 1 - pa] - va - kb;
            }
            const int wmax = __reduce_max_sync(0xffffffffu, cnt);
            double sum = 0.0;
            for (int base = 0; base < wmax; base += CH) {
                double xv[CH], vv[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const bool m = base + u < cnt;
                    const int k = kb + base + u;
                    const int c = m ? cs[k + dc] : 0;
                    vv[u] = m ? vs[k] : 0.0;
                    xv[u] = ldg_keep(xb + c, pol_keep);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (base + u >= wmax) break;   // warp-uniform
                    const double t0 = fma(vv[u], xv[u], sum);
                    sum = (base + u < cnt) ? t0 : sum;
                }
            }
            if (row < d.r1) store_row(a, row, sum);
        }
        __syncwarp();   // stage s is free again
    }
    if (aborted && lane == 0) {
        atomicExch(a.err, kErrTimeout);
        for (int jj = j + 1; jj < j + ST; ++jj) {
            if (first + jj * stride >= tile_end) break;
            mbar_wait_bounded(smem_u32(&bars[w][jj % ST]), (uint32_t)((jj / ST) & 1), kDrainLimitNs);
        }
    }
}

template <int WARPS, int CAP, int ST, int CH>
static cudaError_t run_warp(const CsrArgs& a, const Tile* tiles, int tb, int te, int num_sms, cudaStream_t s) {
    using L = TileLayout<32, CAP>;
    const size_t smem = (size_t)WARPS * ST * L::BYTES;
    static std::atomic<unsigned long long> configured{0};   // one bit per device ordinal
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(configured.load(std::memory_order_acquire) >> dev & 1ull)) {
        e = cudaFuncSetAttribute(csr_warp_kernel<WARPS, CAP, ST, CH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured.fetch_or(1ull << dev, std::memory_order_acq_rel);
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, csr_warp_kernel<WARPS, CAP, ST, CH>, WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int grid = num_sms * occ;
    const int need = (te - tb + WARPS - 1) / WARPS;
    if (grid > need) grid = need;
    return launch_pdl(csr_warp_kernel<WARPS, CAP, ST, CH>, dim3(grid), dim3(WARPS * 32), smem, s, a, tiles, tb, te);
}

// Warp-tile geometries: (warps per CTA, entries per stage, stages, gathers per chunk).
int warp_tile_cap(int param) {
    switch (param) {
        case 0: return 896;    // 32 rows x 28 entries
        case 1: return 896;
        case 2: return 896;
        case 3: return 1792;   // rows up to 56 entries
        case 4: return 896;
        default: return -1;
    }
}

cudaError_t launch_warp(const CsrArgs& a, const Tile* tiles, int tb, int te, int param, int num_sms,
                        cudaStream_t s) {
    if (te <= tb) return cudaSuccess;
    switch (param) {
        case 0: return run_warp<8, 896, 2, 16>(a, tiles, tb, te, num_sms, s);    // 175 KB, 1 CTA
        case 1: return run_warp<4, 896, 2, 16>(a, tiles, tb, te, num_sms, s);    // 88 KB, 2 CTAs
        case 2: return run_warp<10, 896, 2, 16>(a, tiles, tb, te, num_sms, s);   // 219 KB, 1 CTA
        case 3: return run_warp<4, 1792, 2, 16>(a, tiles, tb, te, num_sms, s);   // 174 KB, 1 CTA
        case 4: return run_warp<10, 896, 2, 32>(a, tiles, tb, te, num_sms, s);   // 219 KB, 32 gathers in flight
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------
// Pair-per-lane CSR: V lanes share a row; the row's entries are covered by
// aligned pairs [k, k+1) (k even) and lane h takes pairs h, h+V, h+2V, ...
// Each pair is one 16-byte load of values and one 8-byte load of columns.
// FP64 cost on this part is per warp instruction whatever the active mask,
// so the FMA loop runs exactly as many pairs as the warp's longest share
// (warp-uniform), U pairs of gathers are in flight per lane, and the V
// partial sums meet in a fixed xor-butterfly.  For a 27-entry row and V = 2
// this is 14 FMA instructions + 1 add per 16 rows.
// ------------------------------------------------------------------------
template <int V, int U, int MINB>
__global__ void __launch_bounds__(256, MINB) csr_pair_kernel(CsrArgs a, const Tile* __restrict__ tiles,
                                                          int tile_begin, int tile_end) {
    pdl_begin(a.pdl);  // the previous kernel of this stream is done (unless independent)
    constexpr int GROUPS = 256 / V;
    const uint64_t pol_keep = policy_evict_last();
    const int lane = threadIdx.x % V;
    const int group = threadIdx.x / V;
    for (int t = tile_begin + (int)blockIdx.x; t < tile_end; t += (int)gridDim.x) {
        const Tile d = tiles[t];
        const double* xb = a.x + d.xoff;
        for (int rbase = d.r0; rbase < d.r1; rbase += GROUPS) {
            const int row = rbase + group;
            int kb = 0, ke = 0, k2 = 0, cnt = 0;
            if (row < d.r1) {
                kb = __ldg(a.ptr + row);
                ke = __ldg(a.ptr + row + 1);
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
                    const int k = act ? k2 + 2 * (lane + V * j) : k2;   // k2 is a valid even index
                    vv[u] = __ldg(reinterpret_cast<const double2*>(a.val + k));
                    const int2 c = __ldg(reinterpret_cast<const int2*>(a.col + k));
                    m0[u] = act && k >= kb;
                    m1[u] = act && k + 1 < ke;
                    x0[u] = ldg_keep(xb + (m0[u] ? c.x : 0), pol_keep);
                    x1[u] = ldg_keep(xb + (m1[u] ? c.y : 0), pol_keep);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (j0 + u >= wmax) break;   // warp-uniform
                    double t0 = fma(vv[u].x, x0[u], sum);
                    sum = m0[u] ? t0 : sum;
                    t0 = fma(vv[u].y, x1[u], sum);
                    sum = m1[u] ? t0 : sum;
                }
            }
#pragma unroll
            for (int off = V / 2; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off, V);
            if (row < d.r1 && lane == 0) store_row(a, row, sum);
        }
    }
}

cudaError_t launch_pairs(const CsrArgs& a, const Tile* tiles, int tile_begin, int tile_end, int lanes,
                         int num_sms, cudaStream_t s) {
    if (tile_end <= tile_begin) return cudaSuccess;
    int grid = num_sms * 8;
    if (grid > tile_end - tile_begin) grid = tile_end - tile_begin;
    // lanes 1/2/4/8: 4 pairs in flight per lane (up to 64 registers);
    // 102/104: 2 or 4 lanes with 2 pairs in flight in 32 registers, so 8
    // CTAs (64 warps) fit on an SM
    cudaError_t e = cudaSuccess;
    switch (lanes) {
        case 1: e = launch_pdl(csr_pair_kernel<1, 4, 4>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 2: e = launch_pdl(csr_pair_kernel<2, 4, 4>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 4: e = launch_pdl(csr_pair_kernel<4, 4, 4>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 8: e = launch_pdl(csr_pair_kernel<8, 2, 4>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 102: e = launch_pdl(csr_pair_kernel<2, 2, 8>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 104: e = launch_pdl(csr_pair_kernel<4, 2, 8>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

cudaError_t launch_vector(const CsrArgs& a, const Tile* tiles, int tile_begin, int tile_end,
                          int lanes, int num_sms, cudaStream_t s) {
    if (tile_end <= tile_begin) return cudaSuccess;
    int grid = num_sms * 8;
    if (grid > tile_end - tile_begin) grid = tile_end - tile_begin;
    cudaError_t e = cudaSuccess;
    switch (lanes) {
        case 2: e = launch_pdl(csr_vector_kernel<2>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 4: e = launch_pdl(csr_vector_kernel<4>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 8: e = launch_pdl(csr_vector_kernel<8>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 16: e = launch_pdl(csr_vector_kernel<16>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        case 32: e = launch_pdl(csr_vector_kernel<32>, dim3(grid), dim3(256), 0, s, a, tiles, tile_begin, tile_end); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

// ------------------------------------------------------------------------
// Self-test of the bounded wait: one thread waits on an mbarrier that no
// copy and no thread ever completes; the wait gives up after limit_ns and
// the kernel reports SPMV_ETIMEOUT's magnitude through `status`.
// ------------------------------------------------------------------------
__global__ void selftest_wait_kernel(uint64_t limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns);
        *status = ok ? 0 : kErrTimeout;
    }
}

cudaError_t selftest_wait_timeout(uint64_t limit_ns, int* status_host) {
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return e;
    selftest_wait_kernel<<<1, 32>>>(limit_ns, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(status_host, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}

// ------------------------------------------------------------------------
// FP64 FMA throughput probe: the first `lanes` lanes of every warp run 8
// independent chains of `iters` fused multiply-adds each (enough chains to
// cover the pipe's latency), then store their sum, so no chain is dead code.
// Each chain accumulates through the addend, a = fma(m, c, a), as a product
// accumulates sum = fma(value, x, sum), with every operand a register of its
// own (m and c pass through an opaque move, so they are not folded into
// constant operands).  m c = 1e-6 keeps every value near 1 (no overflow, no
// subnormals).
// ------------------------------------------------------------------------
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__device__ __forceinline__ double opaque(double v) {
    double r;
    asm volatile("mov.b64 %0, %1;" : "=d"(r) : "d"(v));
    return r;
}

__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(int64_t iters, int lanes, double* out) {
    const int64_t gid = (int64_t)blockIdx.x * kProbeThreads + threadIdx.x;
    double a[kProbeChains], m[kProbeChains], c[kProbeChains];
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) {
        a[u] = 1.0 + 1e-3 * u + 1e-9 * (double)(gid & 1023);
        m[u] = opaque(1e-3);
        c[u] = opaque(1e-3);
    }
    if ((int)(threadIdx.x & 31) < lanes) {
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kProbeChains; ++u) a[u] = fma(m[u], c[u], a[u]);
        }
    }
    double sum = 0.0;
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) sum += a[u];
    out[gid] = sum;
}

int probe_threads() { return kProbeThreads; }

cudaError_t launch_dfma_probe(int64_t iters, int grid, int lanes, double* out, int64_t* dfma, cudaStream_t s) {
    dfma_probe_kernel<<<grid, kProbeThreads, 0, s>>>(iters, lanes, out);
    *dfma = (int64_t)grid * (kProbeThreads / 32) * lanes * kProbeChains * iters;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Gather throughput probe: thread g of T sums table[idx[k]] over k = g,
// g + T, g + 2T, ... (four gathers in flight), the access pattern of a
// product's x gathers with the column stream read coalesced; each thread
// stores its sum.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kProbeThreads) gather_probe_kernel(const double* __restrict__ table,
                                                                     const int32_t* __restrict__ idx,
                                                                     int64_t count, double* out) {
    const int64_t T = (int64_t)gridDim.x * kProbeThreads;
    const int64_t g = (int64_t)blockIdx.x * kProbeThreads + threadIdx.x;
    double sum = 0.0;
    int64_t k = g;
    for (; k + 3 * T < count; k += 4 * T) {
        const int32_t i0 = __ldg(idx + k), i1 = __ldg(idx + k + T), i2 = __ldg(idx + k + 2 * T),
                      i3 = __ldg(idx + k + 3 * T);
        const double v0 = __ldg(table + i0), v1 = __ldg(table + i1), v2 = __ldg(table + i2),
                     v3 = __ldg(table + i3);
        sum += v0;
        sum += v1;
        sum += v2;
        sum += v3;
    }
    for (; k < count; k += T) sum += __ldg(table + __ldg(idx + k));
    out[g] = sum;
}

cudaError_t launch_gather_probe(const double* table, const int32_t* idx, int64_t count, int grid, double* out,
                                cudaStream_t s) {
    gather_probe_kernel<<<grid, kProbeThreads, 0, s>>>(table, idx, count, out);
    return cudaGetLastError();
}

}  // namespace spmvk
