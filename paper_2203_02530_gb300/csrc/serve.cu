// Serving runtime: SpMV requests over matrices resident in HBM, with
// continuous batching.
//
// A request names a matrix of a resident batch, a width k (1..8 right-hand
// sides) and a seed; its X (n x k) is drawn on the device from the seed with
// SplitMix64, so no input crosses PCIe/C2C.  The loop runs open-loop against
// the requests' arrival times: arrived requests queue per matrix; whenever a
// stream slot and budget memory are free, the oldest requests of a matrix
// are merged into one multi-RHS block (total width <= 8) and launched; a
// request arriving while blocks run is admitted at the next turn of the
// loop, so blocks of different matrices overlap on the device.  Completion
// is observed through events; latency = observed completion - arrival.
//
// Each column of a block is summed by the same lanes in the same order
// whatever the block's width and partners, so a request's Y is bit-identical
// alone and in any mix (checked through an order-independent 64-bit hash of
// its bits).
#include "batch.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <vector>

using spmvk::BatchMat;
using spmvk::BSlice;

namespace {

constexpr int kMaxW = 8;          // widest block
constexpr int kBatchSliced = 64;  // batch lanes value of the sliced layout
constexpr int kThreads = 256;
constexpr int kMidRow = 256;      // rows up to this length (above the short
                                  // threshold) get 8 lanes, longer rows 32

// ---------------------------------------------------------------- device
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// SplitMix64 (Steele, Lea and Flood) output function; element t of the
// stream of `seed` is splitmix_out(seed + (t + 1) * kGolden).
__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ int clz64(uint64_t a) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)a);
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}

// The IEEE-754 bits of m * 2^-52 - 1 for a 53-bit m (the uniform draw on
// [-1, 1) from the top 53 bits of a SplitMix64 output), built with integer
// operations only.  The value is exact in binary64 (a multiple of 2^-52 of
// magnitude at most 1), so this equals converting m and subtracting; it keeps
// the generator off the FP64 pipe, which the multi-RHS products saturate.
// With a = |m - 2^52| and b its top bit, the value is +-a * 2^-52: the
// significand is a shifted up to bit 52 and the biased exponent 1023 + b - 52;
// a = 0 gives +0.
__host__ __device__ __forceinline__ uint64_t pm1_bits_from_u53(uint64_t m) {
    const int64_t t = (int64_t)m - (int64_t(1) << 52);
    const uint64_t s = (uint64_t)(t >> 63);           // all ones when t < 0
    const uint64_t a = ((uint64_t)t ^ s) - s;         // |t|, at most 2^52
    const int b = 63 - clz64(a);                      // 0 .. 52 when a > 0
    const uint64_t bits = ((a << ((52 - b) & 63)) + ((uint64_t)(970 + b) << 52)) | (s << 63);
    return a ? bits : 0ull;
}

struct BlockReq {
    uint64_t seed;
    int col0;     // first column of the request in the block
    int width;
    int index;    // request index (hash slot)
    int pad;
};

struct BlockDesc {
    BlockReq req[kMaxW];
    int n_req;
    int width;
};

// X[i, c] for every column of every request of a block (row-major, ld W):
// request r's element (i, j) is U(seed_r, 8 i + j), columns of no request 0.
// Thread `tid` of `nthreads` (nthreads >= W) owns column tid mod W and rows
// tid / W, tid / W + R, ... with R = nthreads / W, so consecutive threads
// write consecutive elements and the counter advances by a constant.
__device__ __forceinline__ void gen_x(double* __restrict__ X, int n, int W, const BlockReq* req, int n_req,
                                      int tid, int nthreads) {
    const int R = nthreads / W;
    if (tid >= R * W) return;
    const int c = tid % W;
    int i = tid / W;
    uint64_t seed = 0;
    int j = -1;
    for (int r = 0; r < n_req; ++r) {
        const BlockReq q = req[r];
        if (c >= q.col0 && c < q.col0 + q.width) { seed = q.seed; j = c - q.col0; }
    }
    if (j < 0) {
        for (; i < n; i += R) X[(int64_t)i * W + c] = 0.0;
        return;
    }
    uint64_t z = seed + ((uint64_t)i * kMaxW + (uint64_t)j + 1) * kGolden;
    const uint64_t dz = (uint64_t)R * kMaxW * kGolden;
#pragma unroll 4
    for (; i < n; i += R, z += dz)
        X[(int64_t)i * W + c] = __longlong_as_double((long long)pm1_bits_from_u53(splitmix_out(z) >> 11));
}

__global__ void gen_x_kernel(double* __restrict__ X, int n, BlockDesc b) {
    gen_x(X, n, b.width, b.req, b.n_req, (int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x));
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xFF51AFD7ED558CCDull;
    z = (z ^ (z >> 33)) * 0xC4CEB9FE1A85EC53ull;
    return z ^ (z >> 33);
}

// A row of X (W values, leading dimension W): two per 16-byte load when W
// is even (every row then starts 16-byte aligned), else one at a time.
template <int W>
__device__ __forceinline__ void load_row(const double* xr, double (&xv)[W]) {
    if (W % 2 == 0) {
#pragma unroll
        for (int c = 0; c < W; c += 2) {
            const double2 t = __ldg(reinterpret_cast<const double2*>(xr + c));
            xv[c] = t.x;
            xv[c + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < W; ++c) xv[c] = __ldg(xr + c);
    }
}

// Hash of row `row`'s W values into the per-request sums h (definition below).
template <int W>
__device__ __forceinline__ void hash_row(const BlockReq* req, int n_req, int row, const double (&acc)[W],
                                         unsigned long long (&h)[kMaxW]) {
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) {
        if (r >= n_req) break;
        const BlockReq q = req[r];
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (c >= q.col0 && c < q.col0 + q.width) {
                const uint64_t e = (uint64_t)row * q.width + (uint64_t)(c - q.col0);
                h[r] += mix64((uint64_t)__double_as_longlong(acc[c]) + e * kGolden);
            }
        }
    }
}

__device__ __forceinline__ void flush_hash(const BlockReq* req, int n_req, unsigned long long (&h)[kMaxW],
                                           unsigned long long* hashes) {
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) {
        if (r >= n_req) break;
        unsigned long long v = h[r];
        h[r] = 0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(hashes + req[r].index, v);
    }
}

// Y[:, 0..W) = A X[:, 0..W): V lanes per row, lane h takes entries
// kb + h, kb + h + V, ...; each column accumulates in entry order, then a
// fixed xor-butterfly over the V lanes.
// With `hashes`, every request of the block also gets the order-independent
// hash of its columns: sum (mod 2^64) over its elements (i, j) of
// mix64(bits(y_ij) + (i * width + j) * golden), accumulated per thread and
// added once per warp.
template <int V, int W>
__global__ void __launch_bounds__(kThreads) spmm_kernel(const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ X,
                                                        double* __restrict__ Y, int n, BlockDesc b,
                                                        unsigned long long* __restrict__ hashes,
                                                        int short_max) {
    constexpr int GROUPS = kThreads / V;
    const int lane = threadIdx.x % V;
    unsigned long long h[kMaxW];
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) h[r] = 0;
    for (int rbase = (int)blockIdx.x * GROUPS; rbase < n; rbase += (int)gridDim.x * GROUPS) {
        const int row = rbase + (int)threadIdx.x / V;
        double acc[W];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = 0.0;
        bool mine = row < n;   // rows longer than short_max belong to the bucket kernels
        if (mine) {
            const int kb = __ldg(ptr + row), ke = __ldg(ptr + row + 1);
            mine = ke - kb <= short_max;
            for (int k = kb + lane; mine && k < ke; k += V) {
                const double a = __ldg(val + k);
                const double* xr = X + (int64_t)__ldg(col + k) * W;
                double xv[W];
                load_row<W>(xr, xv);
#pragma unroll
                for (int c = 0; c < W; ++c) acc[c] = fma(a, xv[c], acc[c]);
            }
        }
#pragma unroll
        for (int off = V / 2; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < W; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off, V);
        if (mine && lane == 0) {
#pragma unroll
            for (int c = 0; c < W; ++c) Y[(int64_t)row * W + c] = acc[c];
            if (hashes) hash_row<W>(b.req, b.n_req, row, acc, h);
        }
    }
    if (hashes) flush_hash(b.req, b.n_req, h, hashes);
}

// Rows from a list (one length bucket of a matrix): V lanes per row, lanes
// strided over the row's entries, W accumulators per lane, a fixed
// xor-butterfly; hash as in spmm_kernel.
template <int V, int W>
__global__ void __launch_bounds__(kThreads) spmm_list_kernel(const int32_t* __restrict__ ptr,
                                                             const int32_t* __restrict__ col,
                                                             const double* __restrict__ val,
                                                             const double* __restrict__ X,
                                                             double* __restrict__ Y,
                                                             const int32_t* __restrict__ rows, int n_rows,
                                                             BlockDesc b,
                                                             unsigned long long* __restrict__ hashes) {
    constexpr int GROUPS = kThreads / V;
    const int lane = threadIdx.x % V;
    unsigned long long h[kMaxW];
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) h[r] = 0;
    for (int base = (int)blockIdx.x * GROUPS; base < n_rows; base += (int)gridDim.x * GROUPS) {
        const int wr = base + (int)threadIdx.x / V;
        double acc[W];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = 0.0;
        int row = -1;
        if (wr < n_rows) {
            row = __ldg(rows + wr);
            const int kb = __ldg(ptr + row), ke = __ldg(ptr + row + 1);
            for (int k = kb + lane; k < ke; k += V) {
                const double a = __ldg(val + k);
                const double* xr = X + (int64_t)__ldg(col + k) * W;
                double xv[W];
                load_row<W>(xr, xv);
#pragma unroll
                for (int c = 0; c < W; ++c) acc[c] = fma(a, xv[c], acc[c]);
            }
        }
#pragma unroll
        for (int off = V / 2; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < W; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off, V);
        if (row >= 0 && lane == 0) {
#pragma unroll
            for (int c = 0; c < W; ++c) Y[(int64_t)row * W + c] = acc[c];
            if (hashes) hash_row<W>(b.req, b.n_req, row, acc, h);
        }
    }
    if (hashes) flush_hash(b.req, b.n_req, h, hashes);
}

// One slice of the matrix's sliced layout (the batch's, see
// spmv_batch_set_lanes), Y = A X on its rows: one lane per row, each column
// accumulated in entry order (padded slots discarded by a select), two
// entries' gathers in flight per lane; with `hashes`, the rows' hash terms
// go into h.
template <int W>
__device__ __forceinline__ void sliced_unit(const BatchMat& m, int si, const double* __restrict__ X,
                                            double* __restrict__ Y, const BlockReq* req, int n_req,
                                            unsigned long long* hashes, unsigned long long (&h)[kMaxW]) {
    const int lane = threadIdx.x & 31;
    const BSlice d = m.s_slices[si];
    const int pos = d.pos0 + lane;
    const bool live = lane < d.rows;
    const int len = live ? (int)m.s_len[pos] : 0;
    const double* vp = m.s_val + (int64_t)d.off + lane;
    const int32_t* cp = m.s_col + (int64_t)d.off + lane;
    double acc[W];
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] = 0.0;
    for (int j = 0; j < d.len; j += 2) {
        const int j1 = j + 1 < d.len ? j + 1 : j;
        const double a0 = __ldg(vp + 32 * j), a1 = __ldg(vp + 32 * j1);
        const int c0 = __ldg(cp + 32 * j), c1 = __ldg(cp + 32 * j1);
        double x0[W], x1[W];
        load_row<W>(X + (int64_t)c0 * W, x0);
        load_row<W>(X + (int64_t)c1 * W, x1);
        const bool on0 = j < len, on1 = j + 1 < len;
#pragma unroll
        for (int c = 0; c < W; ++c) {
            const double t = fma(a0, x0[c], acc[c]);
            acc[c] = on0 ? t : acc[c];
        }
        if (j + 1 < d.len) {   // uniform over the warp
#pragma unroll
            for (int c = 0; c < W; ++c) {
                const double t = fma(a1, x1[c], acc[c]);
                acc[c] = on1 ? t : acc[c];
            }
        }
    }
    if (live) {
        const int row = m.s_perm ? __ldg(m.s_perm + pos) : pos;
#pragma unroll
        for (int c = 0; c < W; ++c) Y[(int64_t)row * W + c] = acc[c];
        if (hashes) hash_row<W>(req, n_req, row, acc, h);
    }
}

// The sliced layout's long row at position pos, by the whole warp: lane l
// takes entries l, l+32, ... in order (four in flight), W accumulators
// each, then a fixed xor-butterfly.
template <int W>
__device__ __forceinline__ void long_unit(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, const BatchMat& m, int pos,
                                          const double* __restrict__ X, double* __restrict__ Y,
                                          const BlockReq* req, int n_req, unsigned long long* hashes,
                                          unsigned long long (&h)[kMaxW]) {
    const int lane = threadIdx.x & 31;
    const int row = m.s_perm ? __ldg(m.s_perm + pos) : pos;
    const int kb = __ldg(ptr + row), ke = __ldg(ptr + row + 1);
    double acc[W];
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] = 0.0;
    int k = kb + lane;
    for (; k + 96 < ke; k += 128) {   // four entries per lane in flight
        double a[4], xv[4][W];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = __ldg(val + k + 32 * u);
            load_row<W>(X + (int64_t)__ldg(col + k + 32 * u) * W, xv[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < W; ++c) acc[c] = fma(a[u], xv[u][c], acc[c]);
    }
    for (; k < ke; k += 32) {
        const double a = __ldg(val + k);
        double xv[W];
        load_row<W>(X + (int64_t)__ldg(col + k) * W, xv);
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(a, xv[c], acc[c]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < W; ++c) Y[(int64_t)row * W + c] = acc[c];
        if (hashes) hash_row<W>(req, n_req, row, acc, h);
    }
}

// A long row of more than 2048 entries by the whole CTA: thread t takes
// entries t, t+256, ... in order (four in flight), W accumulators each, a
// fixed xor-butterfly in each warp, then the eight warps' sums added in warp
// order through shared memory; thread 0 stores the row.  All threads of the
// CTA call it for the same row.
template <int W>
__device__ __forceinline__ void long_cta_unit(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                              const double* __restrict__ val, const BatchMat& m, int pos,
                                              const double* __restrict__ X, double* __restrict__ Y,
                                              const BlockReq* req, int n_req, unsigned long long* hashes,
                                              unsigned long long (&h)[kMaxW]) {
    __shared__ double s_part[kThreads / 32][kMaxW];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row = m.s_perm ? __ldg(m.s_perm + pos) : pos;
    const int kb = __ldg(ptr + row), ke = __ldg(ptr + row + 1);
    double acc[W];
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] = 0.0;
    int k = kb + t;
    for (; k + 3 * kThreads < ke; k += 4 * kThreads) {   // four entries per thread in flight
        double a[4], xv[4][W];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = __ldg(val + k + kThreads * u);
            load_row<W>(X + (int64_t)__ldg(col + k + kThreads * u) * W, xv[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < W; ++c) acc[c] = fma(a[u], xv[u][c], acc[c]);
    }
    for (; k < ke; k += kThreads) {
        const double a = __ldg(val + k);
        double xv[W];
        load_row<W>(X + (int64_t)__ldg(col + k) * W, xv);
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(a, xv[c], acc[c]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < W; ++c) s_part[warp][c] = acc[c];
    }
    __syncthreads();
    if (t == 0) {
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = s_part[0][c];
        for (int w = 1; w < kThreads / 32; ++w)
#pragma unroll
            for (int c = 0; c < W; ++c) acc[c] += s_part[w][c];
#pragma unroll
        for (int c = 0; c < W; ++c) Y[(int64_t)row * W + c] = acc[c];
        if (hashes) hash_row<W>(req, n_req, row, acc, h);
    }
    __syncthreads();   // s_part is reused by the CTA's next unit
}

// Long-row work units of a matrix, one per CTA: each of its n_vlong longest
// rows alone, then the other long rows eight at a time, one per warp.
__host__ __device__ __forceinline__ int long_units(const BatchMat& m) {
    return m.n_vlong + (m.n_long - m.n_vlong + kThreads / 32 - 1) / (kThreads / 32);
}

// Long-row unit u of a matrix by the calling CTA (all its threads).
template <int W>
__device__ __forceinline__ void long_units_run(const int32_t* ptr, const int32_t* col, const double* val,
                                               const BatchMat& m, int u, const double* X, double* Y,
                                               const BlockReq* req, int n_req, unsigned long long* hashes,
                                               unsigned long long (&h)[kMaxW]) {
    if (u < m.n_vlong) {
        long_cta_unit<W>(ptr, col, val, m, u, X, Y, req, n_req, hashes, h);
    } else {
        const int pos = m.n_vlong + (u - m.n_vlong) * (kThreads / 32) + (int)(threadIdx.x >> 5);
        if (pos < m.n_long) long_unit<W>(ptr, col, val, m, pos, X, Y, req, n_req, hashes, h);
    }
}

// One block over the sliced layout: one warp per slice (grid-stride).
// Registers capped so that 4 CTAs (widths 1-3) or 3 CTAs (widths 4-8) fit an
// SM without spills; uncapped, width 4 took 128 registers (2 CTAs).
template <int W>
__global__ void __launch_bounds__(kThreads, (W <= 3 ? 4 : 3)) spmm_sliced_kernel(BatchMat m, const double* __restrict__ X,
                                                               double* __restrict__ Y, BlockDesc b,
                                                               unsigned long long* __restrict__ hashes) {
    unsigned long long h[kMaxW];
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) h[r] = 0;
    const int nw = (int)gridDim.x * (kThreads / 32);
    for (int si = (int)blockIdx.x * (kThreads / 32) + (int)(threadIdx.x >> 5); si < m.n_slices; si += nw)
        sliced_unit<W>(m, si, X, Y, b.req, b.n_req, hashes, h);
    if (hashes) flush_hash(b.req, b.n_req, h, hashes);
}

// One block's long rows (positions [0, n_long)): its long-row units, one per
// CTA (grid-stride).
template <int W>
__global__ void __launch_bounds__(kThreads) spmm_long_kernel(const int32_t* __restrict__ ptr,
                                                             const int32_t* __restrict__ col,
                                                             const double* __restrict__ val, BatchMat m,
                                                             const double* __restrict__ X, double* __restrict__ Y,
                                                             BlockDesc b, unsigned long long* __restrict__ hashes) {
    unsigned long long h[kMaxW];
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) h[r] = 0;
    const int units = long_units(m);
    for (int u = (int)blockIdx.x; u < units; u += (int)gridDim.x)
        long_units_run<W>(ptr, col, val, m, u, X, Y, b.req, b.n_req, hashes, h);
    if (hashes) flush_hash(b.req, b.n_req, h, hashes);
}

// ---------------------------------------------------------------- groups
// A group: up to kGroupMax blocks, possibly of different matrices and
// widths, run by one launch per kernel kind.  Block i's X sits at x_off
// (doubles from the pool base), its Y right after (n x width each); its
// slices are the group's units [unit0, next unit0), its long rows the long
// units [long0, next long0).
constexpr int kGroupMax = 64;

struct GroupBlock {
    BlockReq req[kMaxW];
    long long x_off;
    int n_req, width, m, n;
    int unit0, long0, pad0, pad1;
};

__global__ void gen_group_kernel(double* __restrict__ pool, const GroupBlock* __restrict__ g) {
    const GroupBlock& b = g[blockIdx.y];
    gen_x(pool + b.x_off, b.n, b.width, b.req, b.n_req, (int)(blockIdx.x * blockDim.x + threadIdx.x),
          (int)(gridDim.x * blockDim.x));
}

// Units [0, units) of a group, one warp per unit (grid-stride); LONG picks
// the long-row units.  The unit's block is found by binary search over the
// blocks' first units; each unit's hash terms are flushed before the next.
template <bool LONG>
__global__ void __launch_bounds__(kThreads) spmm_group_kernel(const BatchMat* __restrict__ mats,
                                                              const int32_t* __restrict__ ptr,
                                                              const int32_t* __restrict__ col,
                                                              const double* __restrict__ val,
                                                              double* __restrict__ pool,
                                                              const GroupBlock* __restrict__ g, int nb, int units,
                                                              unsigned long long* __restrict__ hashes) {
    __shared__ int s_first[kGroupMax + 1];
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) s_first[i] = i < nb ? (LONG ? g[i].long0 : g[i].unit0) : units;
    __syncthreads();
    unsigned long long h[kMaxW];
#pragma unroll
    for (int r = 0; r < kMaxW; ++r) h[r] = 0;
    // slice units one per warp; long-row units one per CTA (long_units)
    const int nw = LONG ? (int)gridDim.x : (int)gridDim.x * (kThreads / 32);
    const int u0 = LONG ? (int)blockIdx.x : (int)blockIdx.x * (kThreads / 32) + (int)(threadIdx.x >> 5);
    for (int u = u0; u < units; u += nw) {
        int lo = 0, hi = nb - 1;   // the last block whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const GroupBlock& b = g[lo];
        const BatchMat m = mats[b.m];
        double* X = pool + b.x_off;
        double* Y = X + (int64_t)b.n * b.width;
        const int k = u - s_first[lo];
        if (LONG) {
            const int32_t* mp = ptr + m.ptr_off;
            const int32_t* mc = col + m.ent_off;
            const double* mv = val + m.ent_off;
            switch (b.width) {
                case 1: long_units_run<1>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 2: long_units_run<2>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 3: long_units_run<3>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 4: long_units_run<4>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 5: long_units_run<5>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 6: long_units_run<6>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 7: long_units_run<7>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
                default: long_units_run<8>(mp, mc, mv, m, k, X, Y, b.req, b.n_req, hashes, h); break;
            }
        } else {
            switch (b.width) {
                case 1: sliced_unit<1>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 2: sliced_unit<2>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 3: sliced_unit<3>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 4: sliced_unit<4>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 5: sliced_unit<5>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 6: sliced_unit<6>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                case 7: sliced_unit<7>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
                default: sliced_unit<8>(m, k, X, Y, b.req, b.n_req, hashes, h); break;
            }
        }
        if (hashes) flush_hash(b.req, b.n_req, h, hashes);
    }
}

cudaError_t launch_sliced(const BlockDesc& b, const int32_t* ptr, const int32_t* col, const double* val,
                          const BatchMat& M, const double* X, double* Y, int num_sms, unsigned long long* hashes,
                          cudaStream_t s, int64_t& launches) {
    constexpr int WPB = kThreads / 32;
    launches += (M.n_slices > 0) + (M.n_long > 0);
    if (M.n_slices > 0) {
        const int grid = std::min((M.n_slices + WPB - 1) / WPB, num_sms * 8);
#define SPMM_SL(w) spmm_sliced_kernel<w><<<grid, kThreads, 0, s>>>(M, X, Y, b, hashes)
        switch (b.width) {
            case 1: SPMM_SL(1); break;
            case 2: SPMM_SL(2); break;
            case 3: SPMM_SL(3); break;
            case 4: SPMM_SL(4); break;
            case 5: SPMM_SL(5); break;
            case 6: SPMM_SL(6); break;
            case 7: SPMM_SL(7); break;
            default: SPMM_SL(8); break;
        }
#undef SPMM_SL
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (M.n_long > 0) {
        const int grid = std::min(long_units(M), num_sms * 8);
#define SPMM_LG(w) spmm_long_kernel<w><<<grid, kThreads, 0, s>>>(ptr, col, val, M, X, Y, b, hashes)
        switch (b.width) {
            case 1: SPMM_LG(1); break;
            case 2: SPMM_LG(2); break;
            case 3: SPMM_LG(3); break;
            case 4: SPMM_LG(4); break;
            case 5: SPMM_LG(5); break;
            case 6: SPMM_LG(6); break;
            case 7: SPMM_LG(7); break;
            default: SPMM_LG(8); break;
        }
#undef SPMM_LG
    }
    return cudaGetLastError();
}

template <int V>
cudaError_t launch_list_w(const BlockDesc& b, const int32_t* ptr, const int32_t* col, const double* val,
                          const double* X, double* Y, const int32_t* rows, int nr, int num_sms,
                          unsigned long long* hashes, cudaStream_t s) {
    const int grid = std::min((nr + kThreads / V - 1) / (kThreads / V), num_sms * 8);
#define SPMM_LIST(w) spmm_list_kernel<V, w><<<grid, kThreads, 0, s>>>(ptr, col, val, X, Y, rows, nr, b, hashes)
    switch (b.width) {
        case 1: SPMM_LIST(1); break;
        case 2: SPMM_LIST(2); break;
        case 3: SPMM_LIST(3); break;
        case 4: SPMM_LIST(4); break;
        case 5: SPMM_LIST(5); break;
        case 6: SPMM_LIST(6); break;
        case 7: SPMM_LIST(7); break;
        default: SPMM_LIST(8); break;
    }
#undef SPMM_LIST
    return cudaGetLastError();
}

template <int V>
cudaError_t launch_spmm_w(const BlockDesc& b, const int32_t* ptr, const int32_t* col, const double* val,
                          const double* X, double* Y, int n, int grid, unsigned long long* hashes,
                          int short_max, cudaStream_t s) {
#define SPMM_W(w) spmm_kernel<V, w><<<grid, kThreads, 0, s>>>(ptr, col, val, X, Y, n, b, hashes, short_max)
    switch (b.width) {
        case 1: SPMM_W(1); break;
        case 2: SPMM_W(2); break;
        case 3: SPMM_W(3); break;
        case 4: SPMM_W(4); break;
        case 5: SPMM_W(5); break;
        case 6: SPMM_W(6); break;
        case 7: SPMM_W(7); break;
        default: SPMM_W(8); break;
    }
#undef SPMM_W
    return cudaGetLastError();
}

// ---------------------------------------------------------------- pool
// First-fit allocator over one device region: the admission budget.
class Pool {
   public:
    void init(char* base, size_t bytes) {
        base_ = base;
        free_.clear();
        free_[0] = bytes;
        cap_ = bytes;
        used_ = peak_ = 0;
    }
    // offset of a block of `bytes` (rounded to 256), or -1 when none fits
    long long alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return (long long)off;
            }
        }
        return -1;
    }
    void release(long long off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        used_ -= bytes;
        auto it = free_.emplace((size_t)off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char* ptr(long long off) const { return base_ + off; }
    size_t peak() const { return peak_; }
    size_t capacity() const { return cap_; }

   private:
    char* base_ = nullptr;
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace

struct spmv_server {
    spmv_batch* mats = nullptr;
    int n_streams = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<int> lanes;             // lanes per row per matrix
    char* pool_base = nullptr;
    size_t pool_bytes = 0;
    Pool pool;
    unsigned long long* d_hash = nullptr;
    size_t hash_cap = 0;
    int num_sms = 0;
    // per matrix: rows longer than short_max[m] in two buckets (8 lanes up to
    // kMidRow entries, 32 lanes above), as row lists
    std::vector<int> short_max;
    int32_t* bucket_rows = nullptr;
    std::vector<int64_t> mid_off, long_off;   // rows of bucket b of matrix m: [off[m], off[m+1])
    int64_t launches = 0;                      // kernels launched since the last run began
    int group_max = kGroupMax;                 // blocks per group (grouped launches)
    // per stream slot: the group table on the device and its pinned staging
    std::vector<GroupBlock*> d_group, h_group;
};

namespace {

int sfail(int code, const std::string& m) {
    spmvk::set_last_error(m);
    return code;
}

cudaError_t launch_block(spmv_server* sv, int m, const BlockDesc& b, double* X, double* Y,
                         unsigned long long* hashes, cudaStream_t s) {
    spmv_batch* bt = sv->mats;
    const BatchMat& M = bt->mats[m];
    const int n = M.n;
    if (n == 0) return cudaSuccess;
    sv->launches += 2;   // X generator, product over the short rows (or the slices)
    int g = (int)std::min<int64_t>(((int64_t)n * b.width + kThreads - 1) / kThreads, (int64_t)sv->num_sms * 8);
    gen_x_kernel<<<g, kThreads, 0, s>>>(X, n, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int32_t* ptr = bt->ptr + M.ptr_off;
    const int32_t* col = bt->col + M.ent_off;
    const double* val = bt->val + M.ent_off;
    if (M.lanes == kBatchSliced) {
        sv->launches -= 1;
        return launch_sliced(b, ptr, col, val, M, X, Y, sv->num_sms, hashes, s, sv->launches);
    }
    const int V = sv->lanes[m];
    int grid = (int)std::min<int64_t>((n + (kThreads / V) - 1) / (kThreads / V), (int64_t)sv->num_sms * 8);
    const int smax = sv->short_max[m];
    switch (V) {
        case 1: e = launch_spmm_w<1>(b, ptr, col, val, X, Y, n, grid, hashes, smax, s); break;
        case 2: e = launch_spmm_w<2>(b, ptr, col, val, X, Y, n, grid, hashes, smax, s); break;
        case 4: e = launch_spmm_w<4>(b, ptr, col, val, X, Y, n, grid, hashes, smax, s); break;
        default: e = launch_spmm_w<8>(b, ptr, col, val, X, Y, n, grid, hashes, smax, s); break;
    }
    if (e != cudaSuccess) return e;
    const int nm = (int)(sv->mid_off[m + 1] - sv->mid_off[m]);
    const int nl_ = (int)(sv->long_off[m + 1] - sv->long_off[m]);
    sv->launches += (nm > 0) + (nl_ > 0);
    if (nm > 0)
        e = launch_list_w<8>(b, ptr, col, val, X, Y, sv->bucket_rows + sv->mid_off[m], nm, sv->num_sms,
                             hashes, s);
    if (e != cudaSuccess) return e;
    const int nl = (int)(sv->long_off[m + 1] - sv->long_off[m]);
    if (nl > 0)
        e = launch_list_w<32>(b, ptr, col, val, X, Y, sv->bucket_rows + sv->long_off[m], nl, sv->num_sms,
                              hashes, s);
    return e;
}

}  // namespace

#define SERVE_TRY try {
#define SERVE_CATCH                                              \
    }                                                            \
    catch (const spmvk::Fail& f) {                               \
        return sfail(f.code, f.msg);                             \
    }                                                            \
    catch (const std::bad_alloc&) {                              \
        return sfail(SPMV_ENOMEM, "host allocation failed");     \
    }                                                            \
    catch (...) {                                                \
        return sfail(SPMV_EINVAL, "unexpected exception");       \
    }

extern "C" {

int spmv_serve_create(spmv_batch* mats, int n_streams, int64_t budget_bytes, spmv_server** out) {
    if (!out) return sfail(SPMV_EINVAL, "out is NULL");
    *out = nullptr;
    spmv_server* sv = nullptr;
    SERVE_TRY
    if (!mats) spmvk::fail(SPMV_EINVAL, "matrices are NULL");
    if (n_streams < 1 || n_streams > 64) spmvk::fail(SPMV_EINVAL, "n_streams = %d", n_streams);
    const int64_t resident = (int64_t)mats->device_bytes;
    if (budget_bytes <= resident) spmvk::fail(SPMV_ENOMEM, "budget %lld below the resident matrices (%lld)",
                                              (long long)budget_bytes, (long long)resident);
    sv = new spmv_server();
    sv->mats = mats;
    sv->n_streams = n_streams;
    sv->num_sms = mats->num_sms;
    for (int m = 0; m < mats->count; ++m) {
        if (mats->n[m] >= (int64_t(1) << 28)) spmvk::fail(SPMV_EBOUNDS, "matrix %d: n >= 2^28", m);
        const double mean = mats->n[m] ? (double)mats->nnz[m] / (double)mats->n[m] : 0.0;
        sv->lanes.push_back(mean < 6 ? 1 : mean < 24 ? 2 : mean < 64 ? 4 : 8);
    }
    // row buckets of every matrix: rows up to short_max stay with the
    // main kernel, longer rows go to the 8-lane or the 32-lane list
    {
        std::vector<int32_t> hp((size_t)mats->mats.back().ptr_off + mats->n.back() + 1);
        spmvk::check_cuda(cudaMemcpy(hp.data(), mats->ptr, hp.size() * 4, cudaMemcpyDeviceToHost), "row pointers");
        std::vector<int32_t> mid, lng;
        std::vector<int64_t> mid_cnt(mats->count), lng_cnt(mats->count);
        std::vector<std::vector<int32_t>> mid_rows(mats->count), long_rows(mats->count);
        sv->short_max.assign(mats->count, 0);
        for (int m = 0; m < mats->count; ++m) {
            const double mean = mats->n[m] ? (double)mats->nnz[m] / (double)mats->n[m] : 0.0;
            const int smax = std::max(8, (int)(2.0 * mean + 0.5));
            sv->short_max[m] = smax;
            const int32_t* p = hp.data() + mats->mats[m].ptr_off;
            for (int64_t i = 0; i < mats->n[m]; ++i) {
                const int len = p[i + 1] - p[i];
                if (len > kMidRow) long_rows[m].push_back((int32_t)i);
                else if (len > smax) mid_rows[m].push_back((int32_t)i);
            }
        }
        std::vector<int32_t> all;
        sv->mid_off.assign(mats->count + 1, 0);
        sv->long_off.assign(mats->count + 1, 0);
        for (int m = 0; m < mats->count; ++m) {
            sv->mid_off[m] = (int64_t)all.size();
            all.insert(all.end(), mid_rows[m].begin(), mid_rows[m].end());
        }
        sv->mid_off[mats->count] = (int64_t)all.size();
        for (int m = 0; m < mats->count; ++m) {
            sv->long_off[m] = (int64_t)all.size();
            all.insert(all.end(), long_rows[m].begin(), long_rows[m].end());
        }
        sv->long_off[mats->count] = (int64_t)all.size();
        spmvk::check_cuda(cudaMalloc(reinterpret_cast<void**>(&sv->bucket_rows), all.size() * 4 + 16), "row buckets");
        if (!all.empty())
            spmvk::check_cuda(cudaMemcpy(sv->bucket_rows, all.data(), all.size() * 4, cudaMemcpyHostToDevice),
                              "row buckets");
    }
    // the pool holds the X/Y blocks of every block in flight; beyond what
    // the slots can ever hold at once the budget is never used, so it is
    // not taken
    size_t max_block = 0;
    for (int m = 0; m < mats->count; ++m)
        max_block = std::max(max_block, ((size_t)2 * mats->n[m] * kMaxW * sizeof(double) + 255) & ~size_t(255));
    sv->pool_bytes = std::min((size_t)(budget_bytes - resident),
                              std::max<size_t>(4096, max_block * (size_t)n_streams));
    spmvk::check_cuda(cudaMalloc(reinterpret_cast<void**>(&sv->pool_base), sv->pool_bytes), "pool");
    sv->pool.init(sv->pool_base, sv->pool_bytes);
    sv->streams.resize(n_streams);
    sv->events.resize(n_streams);
    sv->d_group.assign(n_streams, nullptr);
    sv->h_group.assign(n_streams, nullptr);
    for (int i = 0; i < n_streams; ++i) {
        spmvk::check_cuda(cudaStreamCreateWithFlags(&sv->streams[i], cudaStreamNonBlocking), "stream");
        spmvk::check_cuda(cudaEventCreateWithFlags(&sv->events[i], cudaEventDisableTiming), "event");
        spmvk::check_cuda(cudaMalloc(reinterpret_cast<void**>(&sv->d_group[i]), kGroupMax * sizeof(GroupBlock)),
                          "group table");
        spmvk::check_cuda(cudaMallocHost(reinterpret_cast<void**>(&sv->h_group[i]), kGroupMax * sizeof(GroupBlock)),
                          "group staging");
    }
    *out = sv;
    sv = nullptr;
    return SPMV_OK;
    }
    catch (const spmvk::Fail& f) {
        if (sv) spmv_serve_destroy(sv);
        return sfail(f.code, f.msg);
    }
    catch (...) {
        if (sv) spmv_serve_destroy(sv);
        return sfail(SPMV_ENOMEM, "server creation failed");
    }
}

int spmv_serve_destroy(spmv_server* sv) {
    if (!sv) return SPMV_OK;
    cudaDeviceSynchronize();
    for (auto s : sv->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : sv->events)
        if (e) cudaEventDestroy(e);
    if (sv->pool_base) cudaFree(sv->pool_base);
    for (auto p : sv->d_group)
        if (p) cudaFree(p);
    for (auto p : sv->h_group)
        if (p) cudaFreeHost(p);
    if (sv->d_hash) cudaFree(sv->d_hash);
    if (sv->bucket_rows) cudaFree(sv->bucket_rows);
    delete sv;
    return SPMV_OK;
}

uint64_t spmv_serve_pm1_bits(uint64_t m) {
    return pm1_bits_from_u53(m & ((uint64_t(1) << 53) - 1));
}

int spmv_serve_set_group_max(spmv_server* sv, int max_blocks) {
    if (!sv) return sfail(SPMV_EINVAL, "server is NULL");
    if (max_blocks < 1 || max_blocks > kGroupMax)
        return sfail(SPMV_EINVAL, "group size " + std::to_string(max_blocks) + " not in [1, 64]");
    sv->group_max = max_blocks;
    return SPMV_OK;
}

int spmv_serve_launches(const spmv_server* sv, int64_t* out) {
    if (!sv || !out) return sfail(SPMV_EINVAL, "NULL argument");
    *out = sv->launches;
    return SPMV_OK;
}

int spmv_serve_single(spmv_server* sv, int matrix, int width, uint64_t seed, double* y_dev,
                      double* x_dev, cudaStream_t s) {
    SERVE_TRY
    if (!sv) spmvk::fail(SPMV_EINVAL, "server is NULL");
    if (matrix < 0 || matrix >= sv->mats->count) spmvk::fail(SPMV_EINVAL, "matrix %d", matrix);
    if (width < 1 || width > kMaxW) spmvk::fail(SPMV_EINVAL, "width %d", width);
    if (!y_dev || !x_dev) spmvk::fail(SPMV_EINVAL, "buffers are NULL");
    BlockDesc b{};
    b.n_req = 1;
    b.width = width;
    b.req[0] = BlockReq{seed, 0, width, 0, 0};
    spmvk::check_cuda(launch_block(sv, matrix, b, x_dev, y_dev, nullptr, s), "single request");
    SERVE_CATCH
    return SPMV_OK;
}

int spmv_serve_run(spmv_server* sv, int64_t n_req, const int32_t* matrix, const int32_t* width,
                   const uint64_t* seed, const double* arrival_s, int mode, double* latency_s,
                   uint64_t* hash_out, int64_t* stats) {
    SERVE_TRY
    if (!sv) spmvk::fail(SPMV_EINVAL, "server is NULL");
    if (n_req < 0 || (n_req > 0 && (!matrix || !width || !seed || !arrival_s || !latency_s)))
        spmvk::fail(SPMV_EINVAL, "request arrays are NULL");
    if (mode != SPMV_SERVE_BATCHED && mode != SPMV_SERVE_PLAIN) spmvk::fail(SPMV_EINVAL, "mode %d", mode);
    const int M = sv->mats->count;
    sv->launches = 0;
    for (int64_t r = 0; r < n_req; ++r) {
        if (matrix[r] < 0 || matrix[r] >= M) spmvk::fail(SPMV_EINVAL, "request %lld: matrix %d", (long long)r, matrix[r]);
        if (width[r] < 1 || width[r] > kMaxW) spmvk::fail(SPMV_EINVAL, "request %lld: width %d", (long long)r, width[r]);
        if (r && arrival_s[r] < arrival_s[r - 1]) spmvk::fail(SPMV_EINVAL, "arrivals must be non-decreasing");
    }
    for (int m = 0; m < M; ++m)
        if ((((size_t)2 * sv->mats->mats[m].n * kMaxW * sizeof(double) + 255) & ~size_t(255)) > sv->pool.capacity())
            spmvk::fail(SPMV_ENOMEM, "matrix %d: one block of it exceeds the budget", m);
    if (hash_out) {
        if ((size_t)n_req > sv->hash_cap) {
            if (sv->d_hash) cudaFree(sv->d_hash);
            sv->d_hash = nullptr;
            spmvk::check_cuda(cudaMalloc(reinterpret_cast<void**>(&sv->d_hash), (size_t)n_req * 8 + 8), "hashes");
            sv->hash_cap = (size_t)n_req;
        }
        spmvk::check_cuda(cudaMemset(sv->d_hash, 0, (size_t)n_req * 8 + 8), "hashes");
    }
    struct Inflight {
        bool busy = false;
        std::vector<int64_t> reqs;
        std::vector<std::pair<long long, size_t>> allocs;   // pool blocks (offset, bytes)
    };
    // grouped launches when every matrix is in the sliced layout: each free
    // slot takes up to kGroupMax blocks (round robin over the matrices) and
    // runs them with one launch per kernel kind
    bool grouped = mode == SPMV_SERVE_BATCHED;
    for (int m = 0; m < M; ++m) grouped = grouped && sv->mats->mats[m].lanes == kBatchSliced;
    std::vector<Inflight> slot(sv->n_streams);
    std::vector<std::deque<int64_t>> pending(M);
    std::vector<int64_t> pend_width(M, 0);   // total width queued per matrix
    // the matrix whose oldest queued request came first (arrival, then
    // request index): queues are served oldest first in both modes
    auto oldest = [&]() {
        int best = -1;
        for (int k = 0; k < M; ++k) {
            if (pending[k].empty()) continue;
            if (best < 0) {
                best = k;
                continue;
            }
            const int64_t a = pending[k].front(), b = pending[best].front();
            if (arrival_s[a] < arrival_s[b] || (arrival_s[a] == arrival_s[b] && a < b)) best = k;
        }
        return best;
    };
    int64_t next = 0, done = 0, blocks = 0, waits_mem = 0, max_inflight = 0, admitted_while_busy = 0;
    const auto t0 = std::chrono::steady_clock::now();
    auto now_s = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    int64_t queued = 0;
    int64_t last_done = 0;
    double last_progress = 0.0;
    while (done < n_req) {
        const double now = now_s();
        if (done != last_done) {
            last_done = done;
            last_progress = now;
        } else if (now - last_progress > 30.0 && next >= n_req) {
            spmvk::fail(SPMV_ETIMEOUT, "no request completed for 30 s");
        }
        // admission of the requests that have arrived
        int busy_now = 0;
        for (auto& sl : slot) busy_now += sl.busy;
        while (next < n_req && arrival_s[next] <= now) {
            pending[matrix[next]].push_back(next);
            pend_width[matrix[next]] += width[next];
            if (busy_now) ++admitted_while_busy;
            ++next;
            ++queued;
        }
        // completions
        for (int i = 0; i < sv->n_streams; ++i) {
            Inflight& sl = slot[i];
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sv->events[i]);
            if (q == cudaErrorNotReady) continue;
            spmvk::check_cuda(q, "block completion");
            const double t = now_s();
            for (int64_t r : sl.reqs) latency_s[r] = t - arrival_s[r];
            done += (int64_t)sl.reqs.size();
            for (auto& a : sl.allocs) sv->pool.release(a.first, a.second);
            sl.busy = false;
            sl.reqs.clear();
            sl.allocs.clear();
        }
        // launches: one block (or one group of blocks) per free slot, the
        // oldest queue first.  Grouping spreads the blocks the queues would
        // form over all the slots (ceil(blocks / slots) per group, at most
        // group_max): while no more blocks wait than there are slots, every
        // block gets a slot of its own (no request waits for another's
        // block); only a longer queue makes groups, which grow with it, so
        // that the launches fall when the GPU is the bottleneck
        if (queued > 0) {
            int per_group = 1;
            if (grouped) {
                int64_t pend_blocks = 0;
                for (int k = 0; k < M; ++k) pend_blocks += (pend_width[k] + kMaxW - 1) / kMaxW;
                per_group = (int)std::min<int64_t>(
                    sv->group_max, std::max<int64_t>(1, (pend_blocks + sv->n_streams - 1) / sv->n_streams));
            }
            for (int i = 0; i < sv->n_streams && queued > 0; ++i) {
                if (slot[i].busy) continue;
                if (grouped && per_group > 1) {
                    GroupBlock* hg = sv->h_group[i];
                    int nb = 0, units = 0, longs = 0, max_elems = 0;
                    bool out_of_memory = false;
                    while (nb < per_group && queued > 0 && !out_of_memory) {
                        const int m = oldest();
                        if (m < 0) break;
                        const BatchMat& Mm = sv->mats->mats[m];
                        auto& q = pending[m];
                        int take = 0, wsum = 0;
                        while (take < (int)q.size() && take < kMaxW && wsum + width[q[take]] <= kMaxW)
                            wsum += width[q[take++]];
                        const size_t bytes = (size_t)2 * Mm.n * wsum * sizeof(double);
                        const long long off = sv->pool.alloc(bytes);
                        if (off < 0) {
                            ++waits_mem;
                            out_of_memory = true;
                            break;
                        }
                        GroupBlock& gb = hg[nb++];
                        gb = GroupBlock{};
                        for (int t = 0, colx = 0; t < take; ++t) {
                            const int64_t r = q.front();
                            gb.req[gb.n_req++] = BlockReq{seed[r], colx, width[r], (int)r, 0};
                            colx += width[r];
                            slot[i].reqs.push_back(r);
                            q.pop_front();
                        }
                        gb.x_off = off / (long long)sizeof(double);
                        gb.width = wsum;
                        gb.m = m;
                        gb.n = Mm.n;
                        gb.unit0 = units;
                        gb.long0 = longs;
                        units += Mm.n_slices;
                        longs += long_units(Mm);
                        max_elems = std::max(max_elems, Mm.n * wsum);
                        queued -= take;
                        pend_width[m] -= wsum;
                        slot[i].allocs.emplace_back(off, bytes);
                        ++blocks;
                    }
                    if (nb == 0) break;   // no memory: wait for completions
                    cudaStream_t st = sv->streams[i];
                    spmvk::check_cuda(cudaMemcpyAsync(sv->d_group[i], hg, (size_t)nb * sizeof(GroupBlock),
                                                      cudaMemcpyHostToDevice, st),
                                      "group table");
                    double* pool = reinterpret_cast<double*>(sv->pool_base);
                    unsigned long long* hs = hash_out ? sv->d_hash : nullptr;
                    const spmv_batch* bt = sv->mats;
                    if (max_elems > 0) {
                        const int gx = std::max(1, std::min((max_elems + kThreads - 1) / kThreads, sv->num_sms * 2));
                        gen_group_kernel<<<dim3(gx, nb), kThreads, 0, st>>>(pool, sv->d_group[i]);
                        ++sv->launches;
                    }
                    if (units > 0) {
                        const int gs = std::min((units + 7) / 8, sv->num_sms * 8);
                        spmm_group_kernel<false><<<gs, kThreads, 0, st>>>(bt->d_mats, bt->ptr, bt->col, bt->val, pool,
                                                                         sv->d_group[i], nb, units, hs);
                        ++sv->launches;
                    }
                    if (longs > 0) {
                        const int gl = std::min(longs, sv->num_sms * 8);   // one CTA per long-row unit
                        spmm_group_kernel<true><<<gl, kThreads, 0, st>>>(bt->d_mats, bt->ptr, bt->col, bt->val, pool,
                                                                        sv->d_group[i], nb, longs, hs);
                        ++sv->launches;
                    }
                    spmvk::check_cuda(cudaGetLastError(), "group launch");
                    spmvk::check_cuda(cudaEventRecord(sv->events[i], st), "event");
                    slot[i].busy = true;
                    if (out_of_memory) break;
                    continue;
                }
                const int m = oldest();
                if (m < 0) break;
                const int n = sv->mats->mats[m].n;
                // the oldest requests of matrix m whose widths sum to <= 8
                auto& q = pending[m];
                int take = 0, wsum = 0;
                while (take < (int)q.size() && take < kMaxW) {
                    const int64_t r = q[take];
                    if (wsum + width[r] > kMaxW) break;
                    wsum += width[r];
                    ++take;
                    if (mode == SPMV_SERVE_PLAIN) break;   // one request per launch
                }
                const size_t bytes = (size_t)2 * n * wsum * sizeof(double);   // X and Y, ld wsum
                const long long off = sv->pool.alloc(bytes);
                if (off < 0) {   // over budget: wait for memory to free up
                    ++waits_mem;
                    break;
                }
                BlockDesc b{};
                std::vector<int64_t> reqs;
                for (int t = 0, col = 0; t < take; ++t) {
                    const int64_t r = q.front();
                    b.req[b.n_req++] = BlockReq{seed[r], col, width[r], (int)r, 0};
                    col += width[r];
                    reqs.push_back(r);
                    q.pop_front();
                }
                b.width = wsum;
                queued -= (int64_t)reqs.size();
                pend_width[m] -= wsum;
                double* X = reinterpret_cast<double*>(sv->pool.ptr(off));
                double* Y = X + (size_t)n * b.width;
                spmvk::check_cuda(launch_block(sv, m, b, X, Y, hash_out ? sv->d_hash : nullptr,
                                               sv->streams[i]),
                                  "block launch");
                spmvk::check_cuda(cudaEventRecord(sv->events[i], sv->streams[i]), "event");
                slot[i].busy = true;
                slot[i].reqs = std::move(reqs);
                slot[i].allocs.emplace_back(off, bytes);
                ++blocks;
            }
        }
        int64_t inflight = 0;
        for (auto& sl : slot) inflight += sl.busy;
        max_inflight = std::max(max_inflight, inflight);
    }
    const double elapsed = now_s();
    if (hash_out && n_req > 0)
        spmvk::check_cuda(cudaMemcpy(hash_out, sv->d_hash, (size_t)n_req * 8, cudaMemcpyDeviceToHost), "hashes");
    if (stats) {
        stats[0] = blocks;
        stats[1] = max_inflight;
        stats[2] = waits_mem;
        stats[3] = (int64_t)sv->pool.peak();
        stats[4] = (int64_t)(elapsed * 1e9);
        stats[5] = admitted_while_busy;
    }
    SERVE_CATCH
    return SPMV_OK;
}

}  // extern "C"
