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

using spmvk::BatchItem;
using spmvk::BSlice;

constexpr int kSliced = 64;   // lanes value selecting the sliced layout

struct BatchArgs {
    const int32_t* ptr;
    const int32_t* col;
    const double* val;
    const BatchMat* mats;
    const BatchItem* items;
    const int* order;         // claim order of the persistent launch
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
// Streamed operands of the sliced layout, read once: not kept in L1.
__device__ __forceinline__ double ld_stream(const double* p) {
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
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

// One lane's slots j .. j + K - 1 of one slice (K <= the slots left in
// it): K value and K column loads, then K gathers, then K FMAs in slot
// order; slots past the lane's row length are discarded by a select.
template <int K>
__device__ __forceinline__ void slice_round(const double* vp, const int32_t* cp, const double* x, int j, int len,
                                            double& sum, uint64_t pol) {
    int32_t c[K];
    double v[K], xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        c[u] = ld_stream(cp + 32 * (j + u));
        v[u] = ld_stream(vp + 32 * (j + u));
    }
#pragma unroll
    for (int u = 0; u < K; ++u) xv[u] = ldg_keep(x + c[u], pol);
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const double t = fma(v[u], xv[u], sum);
        sum = j + u < len ? t : sum;
    }
}

// The same round over two slices at once (2K gathers in flight per lane).
template <int K>
__device__ __forceinline__ void slice_pair_round(const double* vp0, const int32_t* cp0, const double* vp1,
                                                 const int32_t* cp1, const double* x, int j, int len0, int len1,
                                                 double& sum0, double& sum1, uint64_t pol) {
    int32_t c0[K], c1[K];
    double v0[K], v1[K], x0[K], x1[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        c0[u] = ld_stream(cp0 + 32 * (j + u));
        v0[u] = ld_stream(vp0 + 32 * (j + u));
        c1[u] = ld_stream(cp1 + 32 * (j + u));
        v1[u] = ld_stream(vp1 + 32 * (j + u));
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
        x0[u] = ldg_keep(x + c0[u], pol);
        x1[u] = ldg_keep(x + c1[u], pol);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const double t0 = fma(v0[u], x0[u], sum0);
        sum0 = j + u < len0 ? t0 : sum0;
        const double t1 = fma(v1[u], x1[u], sum1);
        sum1 = j + u < len1 ? t1 : sum1;
    }
}

// The r (< 4) slots left of one slice as one round of r.
__device__ __forceinline__ void slice_tail(int r, const double* vp, const int32_t* cp, const double* x, int j,
                                           int len, double& sum, uint64_t pol) {
    switch (r) {
        case 1: slice_round<1>(vp, cp, x, j, len, sum, pol); break;
        case 2: slice_round<2>(vp, cp, x, j, len, sum, pol); break;
        case 3: slice_round<3>(vp, cp, x, j, len, sum, pol); break;
        default: break;
    }
}

// Slices [s0, s1) of a matrix's sliced layout, two at a time: one lane per
// row of each, one FMA per stored entry in storage order (padded slots
// discarded by a select).  Rounds of 4 slots of both slices while both have
// 4 left (8 gathers in flight per lane), then each slice's last slots as one
// round of exactly that many (both slices in one round when their counts
// match, the usual case since slices of a sorted matrix have similar
// lengths): no slot is loaded twice and no gather repeated.
__device__ __forceinline__ void batch_slices(const BatchArgs& a, const BatchMat& m, int s0, int s1, uint64_t pol) {
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const double* x = a.x + m.row_off;
    double* y = a.y + m.row_off;
    // the item's slice descriptors (at most 32), one per lane, loaded at once
    const BSlice mine = s0 + lane < s1 ? m.s_slices[s0 + lane] : BSlice{0, 0, 0, 0};
    auto desc = [&](int i) {
        return BSlice{__shfl_sync(0xffffffffu, mine.pos0, i), __shfl_sync(0xffffffffu, mine.rows, i),
                      __shfl_sync(0xffffffffu, mine.len, i), __shfl_sync(0xffffffffu, mine.off, i)};
    };
    for (int si = s0; si < s1; si += 2) {
        const bool two = si + 1 < s1;
        const BSlice d0 = desc(si - s0);
        const BSlice d1 = two ? desc(si + 1 - s0) : BSlice{0, 0, 0, 0};
        const int len0 = lane < d0.rows ? (int)m.s_len[d0.pos0 + lane] : 0;
        const int len1 = lane < d1.rows ? (int)m.s_len[d1.pos0 + lane] : 0;
        const double* vp0 = m.s_val + (int64_t)d0.off + lane;
        const int32_t* cp0 = m.s_col + (int64_t)d0.off + lane;
        const double* vp1 = m.s_val + (int64_t)d1.off + lane;
        const int32_t* cp1 = m.s_col + (int64_t)d1.off + lane;
        const int lmin = d0.len < d1.len ? d0.len : d1.len;
        double sum0 = 0.0, sum1 = 0.0;
        int j = 0;
        for (; j + U <= lmin; j += U) slice_pair_round<U>(vp0, cp0, vp1, cp1, x, j, len0, len1, sum0, sum1, pol);
        const int r0 = d0.len - j, r1 = d1.len - j;   // warp-uniform
        if (r0 == r1 && r0 > 0) {   // both below U here
            switch (r0) {
                case 1: slice_pair_round<1>(vp0, cp0, vp1, cp1, x, j, len0, len1, sum0, sum1, pol); break;
                case 2: slice_pair_round<2>(vp0, cp0, vp1, cp1, x, j, len0, len1, sum0, sum1, pol); break;
                default: slice_pair_round<3>(vp0, cp0, vp1, cp1, x, j, len0, len1, sum0, sum1, pol); break;
            }
        } else {
            int k = j;
            for (; k + U <= d0.len; k += U) slice_round<U>(vp0, cp0, x, k, len0, sum0, pol);
            slice_tail(d0.len - k, vp0, cp0, x, k, len0, sum0, pol);
            k = j;
            for (; k + U <= d1.len; k += U) slice_round<U>(vp1, cp1, x, k, len1, sum1, pol);
            slice_tail(d1.len - k, vp1, cp1, x, k, len1, sum1, pol);
        }
        if (lane < d0.rows) y[m.s_perm ? __ldg(m.s_perm + d0.pos0 + lane) : d0.pos0 + lane] = sum0;
        if (lane < d1.rows) y[m.s_perm ? __ldg(m.s_perm + d1.pos0 + lane) : d1.pos0 + lane] = sum1;
    }
}

// Long rows at positions [p0, p1) of a matrix's sliced layout, each by the
// whole warp straight from the CSR arrays.
__device__ __forceinline__ void batch_long(const BatchArgs& a, const BatchMat& m, int p0, int p1, uint64_t pol) {
    const int32_t* ptr = a.ptr + m.ptr_off;
    const int32_t* col = a.col + m.ent_off;
    const double* val = a.val + m.ent_off;
    const double* x = a.x + m.row_off;
    double* y = a.y + m.row_off;
    for (int pos = p0; pos < p1; ++pos) {
        const int row = m.s_perm ? __ldg(m.s_perm + pos) : pos;
        const double t = warp_row(col, val, x, __ldg(ptr + row), __ldg(ptr + row + 1), pol);
        if ((threadIdx.x & 31) == 0) y[row] = t;
    }
}

// Items of the CSR modes (kind 0).
__device__ __forceinline__ void batch_item(const BatchArgs& a, int it, uint64_t pol, double* sv,
                                           int32_t* sc) {
    const BatchItem w = a.items[it];
    const BatchMat& m = a.mats[w.m];   // fields read where used
    switch (m.lanes) {
        case 0: batch_rows_staged(a, m, w.a, w.b, pol, sv, sc); break;
        case 1: batch_rows<1>(a, m, w.a, w.b, pol); break;
        case 2: batch_rows<2>(a, m, w.a, w.b, pol); break;
        case 4: batch_rows<4>(a, m, w.a, w.b, pol); break;
        case 8: batch_rows<8>(a, m, w.a, w.b, pol); break;
        case 16: batch_rows<16>(a, m, w.a, w.b, pol); break;
        default: batch_rows<32>(a, m, w.a, w.b, pol); break;
    }
}

// Items of the sliced layout (kinds 1 and 2).
__device__ __forceinline__ void batch_item_sliced(const BatchArgs& a, int it, uint64_t pol) {
    const BatchItem w = a.items[it];
    const BatchMat& m = a.mats[w.m];   // fields read where used
    if (w.kind == 1)
        batch_long(a, m, w.a, w.b, pol);
    else
        batch_slices(a, m, w.a, w.b, pol);
}

// Fill the sliced layout of one matrix from its CSR arrays: one warp per
// slice, one lane per position.
__global__ void __launch_bounds__(256) batch_slice_fill_kernel(const int32_t* __restrict__ ptr,
                                                               const int32_t* __restrict__ col,
                                                               const double* __restrict__ val, BatchMat m,
                                                               double* __restrict__ s_val,
                                                               int32_t* __restrict__ s_col) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)gridDim.x * 8;
    for (int si = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); si < m.n_slices; si += nw) {
        const BSlice d = m.s_slices[si];
        const int pos = d.pos0 + lane;
        const bool live = lane < d.rows;
        const int row = live ? (m.s_perm ? m.s_perm[pos] : pos) : 0;
        const int kb = live ? ptr[row] : 0;
        const int len = live ? ptr[row + 1] - kb : 0;
        for (int j = 0; j < d.len; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            s_val[o] = j < len ? val[kb + j] : 0.0;
            s_col[o] = j < len ? col[kb + j] : 0;
        }
    }
}

// The inverse of batch_slice_fill_kernel: the live slots of every slice of
// one matrix back into its CSR rows (ptr: the matrix's full row pointers).
__global__ void __launch_bounds__(256) batch_slice_unfill_kernel(const int32_t* __restrict__ ptr, BatchMat m,
                                                                 const double* __restrict__ s_val,
                                                                 const int32_t* __restrict__ s_col,
                                                                 int32_t* __restrict__ col, double* __restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)gridDim.x * 8;
    for (int si = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); si < m.n_slices; si += nw) {
        const BSlice d = m.s_slices[si];
        const int pos = d.pos0 + lane;
        const bool live = lane < d.rows;
        const int row = live ? (m.s_perm ? m.s_perm[pos] : pos) : 0;
        const int kb = live ? ptr[row] : 0;
        const int len = live ? (int)m.s_len[pos] : 0;
        for (int j = 0; j < len; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            val[kb + j] = s_val[o];
            col[kb + j] = s_col[o];
        }
    }
}

// Moves of entry ranges between two CSR arrays: segment s (one warp) copies
// tab[3s + 2] entries from position tab[3s] of (sv, sc) to tab[3s + 1] of
// (dv, dc) (64-bit positions).
__global__ void __launch_bounds__(256) batch_segment_copy_kernel(const int64_t* __restrict__ tab, int64_t n_seg,
                                                                 const double* __restrict__ sv,
                                                                 const int32_t* __restrict__ sc,
                                                                 double* __restrict__ dv, int32_t* __restrict__ dc) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t g = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); g < n_seg; g += nw) {
        const int64_t src = tab[3 * g], dst = tab[3 * g + 1], len = tab[3 * g + 2];
        for (int64_t i = lane; i < len; i += 32) {
            dv[dst + i] = sv[src + i];
            dc[dst + i] = sc[src + i];
        }
    }
}

// Persistent: every warp claims whole items (order[0 .. n_items)) with an
// atomic ticket until none is left (no block-wide barrier: warps never wait
// for each other).  One kernel for the CSR modes (shared-memory slices for
// the staged mode), one for the sliced layout (no shared memory).
__global__ void __launch_bounds__(kThreads, 4) batch_persistent_kernel(BatchArgs a) {
    __shared__ double s_val[kThreads / 32][kStageEntries];
    __shared__ int32_t s_col[kThreads / 32][kStageEntries];
    const uint64_t pol = policy_evict_last();
    const int w = threadIdx.x >> 5;
    for (;;) {
        int t = 0;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(a.ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.n_items) break;
        batch_item(a, __ldg(a.order + t), pol, s_val[w], s_col[w]);
    }
}

__global__ void __launch_bounds__(kThreads, 6) batch_sliced_persistent_kernel(BatchArgs a) {
    const uint64_t pol = policy_evict_last();
    for (;;) {
        int t = 0;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(a.ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.n_items) break;
        batch_item_sliced(a, __ldg(a.order + t), pol);
    }
}

// Items [first, last) of one matrix, one per warp, grid-stride.
__global__ void __launch_bounds__(kThreads, 4) batch_range_kernel(BatchArgs a, int first, int last) {
    __shared__ double s_val[kThreads / 32][kStageEntries];
    __shared__ int32_t s_col[kThreads / 32][kStageEntries];
    const uint64_t pol = policy_evict_last();
    const int w = threadIdx.x >> 5;
    const int nw = (int)gridDim.x * (kThreads / 32);
    for (int it = first + (int)blockIdx.x * (kThreads / 32) + w; it < last; it += nw)
        batch_item(a, it, pol, s_val[w], s_col[w]);
}

__global__ void __launch_bounds__(kThreads, 4) batch_sliced_range_kernel(BatchArgs a, int first, int last) {
    const uint64_t pol = policy_evict_last();
    const int nw = (int)gridDim.x * (kThreads / 32);
    for (int it = first + (int)blockIdx.x * (kThreads / 32) + (int)(threadIdx.x >> 5); it < last; it += nw)
        batch_item_sliced(a, it, pol);
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

void brelease(spmv_batch* b, void* p, size_t bytes) {
    for (size_t i = 0; i < b->allocs.size(); ++i)
        if (b->allocs[i] == p) {
            cudaFree(p);
            b->allocs.erase(b->allocs.begin() + (long)i);
            b->device_bytes -= bytes + 256;
            return;
        }
}

// Item table of the current modes: each matrix's CSR or sliced items, and
// the claim order of the persistent launch (items of long rows first: they
// are the heaviest, so they do not end up in the tail).
void upload_items(spmv_batch* b) {
    std::vector<BatchItem> all;
    std::vector<int64_t> cost;   // estimated work per item (entries plus 8 per row)
    b->item_off.assign(b->count + 1, 0);
    for (int m = 0; m < b->count; ++m) {
        b->item_off[m] = (int)all.size();
        const bool sl = b->mats[m].lanes == kSliced;
        const auto& src = sl ? b->sliced_items[m] : b->csr_items[m];
        const auto& cst = sl ? b->sliced_cost[m] : b->csr_cost[m];
        all.insert(all.end(), src.begin(), src.end());
        cost.insert(cost.end(), cst.begin(), cst.end());
    }
    b->item_off[b->count] = (int)all.size();
    // claim order: matrix by matrix, so that the warps in flight share a
    // few matrices' x in L2 (taking heavy items of every matrix first would
    // spread the gathers over all of them); within a matrix its heaviest
    // items (the long rows) first, so they do not end up in the tail
    b->order.clear();
    for (int i = 0; i < (int)all.size(); ++i)
        if (all[i].kind != 0) b->order.push_back(i);
    b->n_sliced_items = (int)b->order.size();
    for (int i = 0; i < (int)all.size(); ++i)
        if (all[i].kind == 0) b->order.push_back(i);
    auto first = [&](int p, int q) {
        if (all[p].m != all[q].m) return all[p].m < all[q].m;
        return cost[p] > cost[q];
    };
    std::stable_sort(b->order.begin(), b->order.begin() + b->n_sliced_items, first);
    std::stable_sort(b->order.begin() + b->n_sliced_items, b->order.end(), first);
    // where each matrix's items start in either part of the order (the
    // host-buffer path claims one run of matrices at a time)
    b->order_off.assign(2 * (b->count + 1), 0);
    for (int part = 0; part < 2; ++part) {
        const int lo = part == 0 ? 0 : b->n_sliced_items, hi = part == 0 ? b->n_sliced_items : (int)all.size();
        int t = lo;
        for (int m = 0; m <= b->count; ++m) {
            while (t < hi && all[b->order[t]].m < m) ++t;
            b->order_off[part * (b->count + 1) + m] = t;
        }
    }
    // the whole-batch launch takes the sliced items of the length-sorted
    // matrices (skewed rows: bound by their scattered x gathers) and of the
    // natural-order ones (stencils: bound by streaming from HBM) side by
    // side, each run advancing at the same share of its estimated work, so
    // that the two bounds overlap instead of following each other (256-matrix
    // mix: 864 us against 894 us; weighting the gather-bound work 1.6 or 2
    // times made no difference); each run keeps the matrix-by-matrix order
    // above, and the host-buffer path keeps that order itself
    std::vector<int> full(b->order.begin(), b->order.end());
    {
        std::vector<int> ga, st;
        double ca = 0.0, cs = 0.0;
        for (int t = 0; t < b->n_sliced_items; ++t) {
            const int i = b->order[t];
            if (b->mats[all[i].m].s_perm) {
                ga.push_back(i);
                ca += (double)cost[i];
            } else {
                st.push_back(i);
                cs += (double)cost[i];
            }
        }
        if (!ga.empty() && !st.empty()) {
            size_t ia = 0, is = 0, t = 0;
            double da = 0.0, ds = 0.0;
            while (ia < ga.size() || is < st.size()) {
                const bool take_a = is >= st.size() || (ia < ga.size() && da * cs <= ds * ca);
                const int i = take_a ? ga[ia++] : st[is++];
                (take_a ? da : ds) += (double)cost[i];
                full[t++] = i;
            }
        }
    }
    if (all.size() > b->items_cap) {
        if (b->d_items) brelease(b, b->d_items, b->items_cap * sizeof(BatchItem));
        if (b->d_order) brelease(b, b->d_order, b->items_cap * sizeof(int));
        if (b->d_order_full) brelease(b, b->d_order_full, b->items_cap * sizeof(int));
        b->items_cap = all.size();
        b->d_items = balloc(b, b->items_cap * sizeof(BatchItem));
        b->d_order = static_cast<int*>(balloc(b, b->items_cap * sizeof(int)));
        b->d_order_full = static_cast<int*>(balloc(b, b->items_cap * sizeof(int)));
    }
    b->n_items = (int)all.size();
    if (!all.empty()) {
        spmvk::check_cuda(cudaMemcpy(b->d_items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice),
                          "items");
        spmvk::check_cuda(cudaMemcpy(b->d_order, b->order.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice),
                          "item order");
        spmvk::check_cuda(cudaMemcpy(b->d_order_full, full.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice),
                          "item order");
    }
}

// Sliced layout of matrix m.  Natural row order when no row is longer than
// kLongRow and padding to each 32-row slice's longest row adds at most 1/8;
// otherwise rows sorted by length (descending, stable), the rows longer than
// kLongRow first (summed by whole warps), the rest in slices of similar
// lengths.  Items: up to 32 long rows or 4096 of their entries, 8 slices.
void build_sliced(spmv_batch* b, int m) {
    BatchMat& M = b->mats[m];
    const int n = M.n;
    std::vector<int32_t> hp((size_t)n + 1, 0);
    if (n > 0)
        spmvk::check_cuda(cudaMemcpy(hp.data(), b->ptr + M.ptr_off, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost),
                          "row pointers");
    std::vector<int32_t> len((size_t)n);
    for (int i = 0; i < n; ++i) len[i] = hp[i + 1] - hp[i];
    const int64_t nnz = hp[n];
    bool natural = true;
    int64_t padded = 0;
    for (int r = 0; r < n; r += 32) {
        int mx = 0;
        for (int i = r; i < std::min(n, r + 32); ++i) mx = std::max(mx, len[i]);
        if (mx > kLongRow) natural = false;
        padded += 32 * (int64_t)mx;
    }
    if (padded > nnz + nnz / 8 + 1024) natural = false;
    std::vector<int32_t> perm;
    int n_long = 0;
    if (!natural) {
        perm.resize((size_t)n);
        for (int i = 0; i < n; ++i) perm[i] = i;
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t p, int32_t q) { return len[p] > len[q]; });
        while (n_long < n && len[perm[n_long]] > kLongRow) ++n_long;
    }
    auto L = [&](int pos) { return len[natural ? pos : perm[pos]]; };
    std::vector<BSlice> sl;
    std::vector<uint8_t> slen((size_t)n, 0);
    int64_t off = 0;
    for (int p0 = n_long; p0 < n; p0 += 32) {
        const int e = std::min(n, p0 + 32);
        int mx = 0;
        for (int pos = p0; pos < e; ++pos) {
            slen[pos] = (uint8_t)L(pos);
            mx = std::max(mx, L(pos));
        }
        if (off + 32 * (int64_t)mx > INT32_MAX - 64) spmvk::fail(SPMV_EBOUNDS, "matrix %d: sliced layout too large", m);
        sl.push_back(BSlice{p0, e - p0, mx, (int32_t)off});
        off += 32 * (int64_t)mx;
    }
    double* s_val = static_cast<double*>(balloc(b, (size_t)off * 8));
    int32_t* s_col = static_cast<int32_t*>(balloc(b, (size_t)off * 4));
    uint8_t* s_len = static_cast<uint8_t*>(balloc(b, (size_t)n));
    BSlice* s_sl = static_cast<BSlice*>(balloc(b, sl.size() * sizeof(BSlice)));
    int32_t* s_perm = nullptr;
    if (n > 0) spmvk::check_cuda(cudaMemcpy(s_len, slen.data(), (size_t)n, cudaMemcpyHostToDevice), "lengths");
    if (!sl.empty())
        spmvk::check_cuda(cudaMemcpy(s_sl, sl.data(), sl.size() * sizeof(BSlice), cudaMemcpyHostToDevice), "slices");
    if (!natural) {
        s_perm = static_cast<int32_t*>(balloc(b, (size_t)n * 4));
        spmvk::check_cuda(cudaMemcpy(s_perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice), "row order");
    }
    M.s_val = s_val;
    M.s_col = s_col;
    M.s_len = s_len;
    M.s_perm = s_perm;
    M.s_slices = s_sl;
    M.n_long = n_long;
    M.n_vlong = 0;   // long rows come longest first
    while (M.n_vlong < n_long && L(M.n_vlong) > 2048) ++M.n_vlong;
    M.n_slices = (int)sl.size();
    if (!sl.empty()) {
        int grid = ((int)sl.size() + 7) / 8;
        if (grid > b->num_sms * 8) grid = b->num_sms * 8;
        batch_slice_fill_kernel<<<grid, 256>>>(b->ptr + M.ptr_off, b->col + M.ent_off, b->val + M.ent_off, M,
                                               s_val, s_col);
        spmvk::check_cuda(cudaGetLastError(), "sliced fill");
        spmvk::check_cuda(cudaDeviceSynchronize(), "sliced fill");
    }
    std::vector<BatchItem>& items = b->sliced_items[m];
    std::vector<int64_t>& cost = b->sliced_cost[m];
    items.clear();
    cost.clear();
    for (int p = 0; p < n_long;) {   // up to 32 long rows or 4096 of their entries
        int e = p;
        int64_t ent = 0;
        while (e < n_long && e - p < 32 && ent < 4096) ent += L(e++);
        items.push_back(BatchItem{m, 1, p, e});
        cost.push_back(ent + ent / 2 + 8 * (e - p));
        p = e;
    }
    for (int s0 = 0; s0 < (int)sl.size();) {   // up to 8 slices or 4096 padded slots
        int s1 = s0;
        int64_t slots = 0;
        while (s1 < (int)sl.size() && s1 - s0 < 8 && slots < 4096) slots += 32 * (int64_t)sl[s1++].len;
        items.push_back(BatchItem{m, 2, s0, s1});
        cost.push_back(slots + 8 * 32 * (int64_t)(s1 - s0));
        s0 = s1;
    }
    b->sliced_built[m] = 1;
}

template <class T>
std::vector<T> bdownload(const T* d, size_t count) {
    std::vector<T> h(count);
    if (count) spmvk::check_cuda(cudaMemcpy(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost), "download");
    return h;
}

void run_segment_copy(spmv_batch* b, const std::vector<int64_t>& tab, const double* sv, const int32_t* sc, double* dv,
                      int32_t* dc) {
    const int64_t n_seg = (int64_t)tab.size() / 3;
    if (n_seg == 0) return;
    int64_t* d_tab = static_cast<int64_t*>(balloc(b, tab.size() * sizeof(int64_t)));
    spmvk::check_cuda(cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "segments");
    const int64_t grid = std::min<int64_t>((n_seg + 7) / 8, (int64_t)b->num_sms * 8);
    batch_segment_copy_kernel<<<(unsigned)grid, 256>>>(d_tab, n_seg, sv, sc, dv, dc);
    spmvk::check_cuda(cudaGetLastError(), "segment copy");
    spmvk::check_cuda(cudaDeviceSynchronize(), "segment copy");
    brelease(b, d_tab, tab.size() * sizeof(int64_t));
}

// Release of the CSR copy of a batch whose matrices all use the sliced
// layout: only the rows longer than kLongRow (which the sliced products read
// from the CSR) stay, in compact arrays whose row pointers give every other
// row zero length, so every reader of a long row finds it where it looks.
void batch_release_csr(spmv_batch* b) {
    if (b->csr_released) return;
    for (int m = 0; m < b->count; ++m)
        if (b->mats[m].lanes != kSliced || !b->sliced_built[m])
            spmvk::fail(SPMV_EINVAL, "matrix %d does not use the sliced layout: the CSR copy is still read", m);
    spmvk::check_cuda(cudaDeviceSynchronize(), "synchronize");
    const size_t ptr_total = (size_t)(b->mats.back().ptr_off + b->n.back() + 1);
    b->h_full_ptr = bdownload(b->ptr, ptr_total);
    b->full_ent_off.resize(b->count);
    std::vector<int32_t> cptr(ptr_total, 0);
    std::vector<long long> ent_off(b->count);
    std::vector<int64_t> tab;
    long long ent = 0;
    for (int m = 0; m < b->count; ++m) {
        const BatchMat& M = b->mats[m];
        b->full_ent_off[m] = M.ent_off;
        const int32_t* fp = b->h_full_ptr.data() + M.ptr_off;
        int32_t* cp = cptr.data() + M.ptr_off;
        for (int i = 0; i < M.n; ++i) {
            const int32_t len = fp[i + 1] - fp[i];
            const bool keep = len > kLongRow;
            cp[i + 1] = cp[i] + (keep ? len : 0);
            if (keep) {
                tab.push_back(M.ent_off + fp[i]);
                tab.push_back(ent + cp[i]);
                tab.push_back(len);
            }
        }
        ent_off[m] = ent;
        ent += ((long long)cp[M.n] + 3) & ~3LL;
    }
    b->full_entries = b->full_ent_off.back() + ((b->nnz.back() + 3) & ~int64_t(3));
    int32_t* nptr = static_cast<int32_t*>(balloc(b, ptr_total * 4));
    int32_t* ncol = static_cast<int32_t*>(balloc(b, (size_t)std::max<long long>(ent, 4) * 4));
    double* nval = static_cast<double*>(balloc(b, (size_t)std::max<long long>(ent, 4) * 8));
    spmvk::check_cuda(cudaMemcpy(nptr, cptr.data(), ptr_total * 4, cudaMemcpyHostToDevice), "row pointers");
    run_segment_copy(b, tab, b->val, b->col, nval, ncol);
    brelease(b, b->ptr, ptr_total * 4);
    brelease(b, b->col, (size_t)b->full_entries * 4);
    brelease(b, b->val, (size_t)b->full_entries * 8);
    b->ptr = nptr;
    b->col = ncol;
    b->val = nval;
    for (int m = 0; m < b->count; ++m) b->mats[m].ent_off = ent_off[m];
    spmvk::check_cuda(cudaMemcpy(b->d_mats, b->mats.data(), b->mats.size() * sizeof(BatchMat), cudaMemcpyHostToDevice),
                      "matrix table");
    b->csr_released = true;
}

// The rebuild: full arrays again, the slices' slots back into their rows and
// the long rows copied back from the compact arrays.
void batch_restore_csr(spmv_batch* b) {
    if (!b->csr_released) return;
    spmvk::check_cuda(cudaDeviceSynchronize(), "synchronize");
    const size_t ptr_total = b->h_full_ptr.size();
    const std::vector<int32_t> cptr = bdownload(b->ptr, ptr_total);
    int32_t* fptr = static_cast<int32_t*>(balloc(b, ptr_total * 4));
    int32_t* fcol = static_cast<int32_t*>(balloc(b, (size_t)b->full_entries * 4));
    double* fval = static_cast<double*>(balloc(b, (size_t)b->full_entries * 8));
    spmvk::check_cuda(cudaMemcpy(fptr, b->h_full_ptr.data(), ptr_total * 4, cudaMemcpyHostToDevice), "row pointers");
    std::vector<int64_t> tab;
    for (int m = 0; m < b->count; ++m) {
        const BatchMat& M = b->mats[m];
        if (M.n_slices > 0) {
            int grid = (M.n_slices + 7) / 8;
            if (grid > b->num_sms * 8) grid = b->num_sms * 8;
            batch_slice_unfill_kernel<<<grid, 256>>>(fptr + M.ptr_off, M, M.s_val, M.s_col, fcol + b->full_ent_off[m],
                                                     fval + b->full_ent_off[m]);
            spmvk::check_cuda(cudaGetLastError(), "slots back into the CSR");
        }
        const int32_t* fp = b->h_full_ptr.data() + M.ptr_off;
        const int32_t* cp = cptr.data() + M.ptr_off;
        for (int i = 0; i < M.n; ++i)
            if (cp[i + 1] > cp[i]) {
                tab.push_back(M.ent_off + cp[i]);
                tab.push_back(b->full_ent_off[m] + fp[i]);
                tab.push_back(cp[i + 1] - cp[i]);
            }
    }
    spmvk::check_cuda(cudaDeviceSynchronize(), "slots back into the CSR");
    run_segment_copy(b, tab, b->val, b->col, fval, fcol);
    const long long ent = b->mats.back().ent_off + (((long long)cptr[(size_t)(b->mats.back().ptr_off + b->n.back())] + 3) & ~3LL);
    brelease(b, b->ptr, ptr_total * 4);
    brelease(b, b->col, (size_t)std::max<long long>(ent, 4) * 4);
    brelease(b, b->val, (size_t)std::max<long long>(ent, 4) * 8);
    b->ptr = fptr;
    b->col = fcol;
    b->val = fval;
    for (int m = 0; m < b->count; ++m) b->mats[m].ent_off = b->full_ent_off[m];
    spmvk::check_cuda(cudaMemcpy(b->d_mats, b->mats.data(), b->mats.size() * sizeof(BatchMat), cudaMemcpyHostToDevice),
                      "matrix table");
    b->h_full_ptr.clear();
    b->full_ent_off.clear();
    b->csr_released = false;
}

BatchArgs args_of(spmv_batch* b, const double* x, double* y) {
    BatchArgs a{};
    a.ptr = b->ptr;
    a.col = b->col;
    a.val = b->val;
    a.mats = b->d_mats;
    a.items = static_cast<const BatchItem*>(b->d_items);
    a.order = b->d_order;
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

namespace {

// The host-buffer path's device vectors and events, made on first use:
// 2 events per chunk (x arrived, y computed), then x free and y free for each
// pair of device vectors of the streamed path.
void batch_host_setup(spmv_batch* b) {
    if (!b->io_x) {
        b->io_x = static_cast<double*>(balloc(b, (size_t)b->total_rows * sizeof(double)));
        b->io_y = static_cast<double*>(balloc(b, (size_t)b->total_rows * sizeof(double)));
        b->io_tickets = static_cast<int*>(balloc(b, 4 * 64 * sizeof(int)));
    }
    while ((int)b->io_ev.size() < 2 * 64 + 4) {
        cudaEvent_t e;
        spmvk::check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        b->io_ev.push_back(e);
    }
}

// One batched product through host buffers and the device vectors xd / yd,
// nothing waited for on the host.  With slot >= 0 it is one of a stream of
// products on two pairs of device vectors: its copies in wait until the
// products that read the same pair's previous x are done, and its products
// until the same pair's previous y has gone out (all products run on
// s_compute, so the chunk tickets are reset after the previous product).
void batch_host_product(spmv_batch* b, const double* x_host, double* y_host, double* xd, double* yd, int chunks,
                        cudaStream_t s_in, cudaStream_t s_compute, cudaStream_t s_out, int slot) {
    cudaEvent_t x_free = slot >= 0 ? b->io_ev[2 * 64 + slot] : nullptr;
    cudaEvent_t y_free = slot >= 0 ? b->io_ev[2 * 64 + 2 + slot] : nullptr;
    // chunks of whole matrices with about equal rows: x of chunk c goes in
    // on s_in, its products run on s_compute once it has arrived, and its y
    // goes back on s_out while later chunks are still moving or computing.
    // Issued phase by phase (all copies in, all products, all copies out) so
    // that streams sharing a hardware queue never hold a copy behind a wait.
    const BatchArgs a = args_of(b, xd, yd);
    struct Chunk {
        int m0, m1;
        long long r0, r1;
    };
    std::vector<Chunk> ch;
    for (int c = 0, m0 = 0; c < chunks && m0 < b->count; ++c) {
        const long long target = b->total_rows * (long long)(c + 1) / chunks;
        int m1 = m0 + 1;
        while (m1 < b->count && b->mats[m1 - 1].row_off + b->n[m1 - 1] < target) ++m1;
        if (c == chunks - 1) m1 = b->count;
        ch.push_back(Chunk{m0, m1, b->mats[m0].row_off, b->mats[m1 - 1].row_off + b->n[m1 - 1]});
        m0 = m1;
    }
    if (x_free) spmvk::check_cuda(cudaStreamWaitEvent(s_in, x_free, 0), "wait");
    for (size_t c = 0; c < ch.size(); ++c) {
        if (ch[c].r1 > ch[c].r0)
            spmvk::check_cuda(cudaMemcpyAsync(xd + ch[c].r0, x_host + ch[c].r0,
                                              (size_t)(ch[c].r1 - ch[c].r0) * sizeof(double),
                                              cudaMemcpyHostToDevice, s_in),
                              "copy x in");
        spmvk::check_cuda(cudaEventRecord(b->io_ev[2 * c], s_in), "event");
    }
    // each chunk's items are a contiguous run of the claim order (per
    // layout), run by the persistent kernels with a ticket of their own
    if (y_free) spmvk::check_cuda(cudaStreamWaitEvent(s_compute, y_free, 0), "wait");
    spmvk::check_cuda(cudaMemsetAsync(b->io_tickets, 0, (size_t)4 * ch.size() * sizeof(int), s_compute),
                      "chunk tickets");
    const int cp1 = b->count + 1;
    for (size_t c = 0; c < ch.size(); ++c) {
        spmvk::check_cuda(cudaStreamWaitEvent(s_compute, b->io_ev[2 * c], 0), "wait");
        for (int part = 0; part < 2; ++part) {
            const int o0 = b->order_off[part * cp1 + ch[c].m0], o1 = b->order_off[part * cp1 + ch[c].m1];
            if (o1 <= o0) continue;
            BatchArgs pa = a;
            pa.order = b->d_order + o0;
            pa.n_items = o1 - o0;
            pa.ticket = b->io_tickets + 4 * c + 2 * part;
            int grid = b->num_sms * std::max(1, part == 0 ? b->occupancy_sliced : b->occupancy);
            const int need = (o1 - o0 + kThreads / 32 - 1) / (kThreads / 32);
            if (grid > need) grid = need;
            if (part == 0)
                batch_sliced_persistent_kernel<<<grid, kThreads, 0, s_compute>>>(pa);
            else
                batch_persistent_kernel<<<grid, kThreads, 0, s_compute>>>(pa);
            spmvk::check_cuda(cudaGetLastError(), "chunk launch");
        }
        spmvk::check_cuda(cudaEventRecord(b->io_ev[2 * c + 1], s_compute), "event");
    }
    if (x_free) spmvk::check_cuda(cudaEventRecord(x_free, s_compute), "event");
    for (size_t c = 0; c < ch.size(); ++c) {
        spmvk::check_cuda(cudaStreamWaitEvent(s_out, b->io_ev[2 * c + 1], 0), "wait");
        if (ch[c].r1 > ch[c].r0)
            spmvk::check_cuda(cudaMemcpyAsync(y_host + ch[c].r0, yd + ch[c].r0,
                                              (size_t)(ch[c].r1 - ch[c].r0) * sizeof(double),
                                              cudaMemcpyDeviceToHost, s_out),
                              "copy y out");
    }
    if (y_free) spmvk::check_cuda(cudaEventRecord(y_free, s_out), "event");
}

}  // namespace

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
    spmvk::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occupancy_sliced,
                                                                    batch_sliced_persistent_kernel, kThreads, 0),
                      "occupancy");
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
        b->mats[m].n_vlong = 0;
        ptr_total += n[m] + 1;
        ent_total += (z + 3) & ~int64_t(3);   // keep every matrix 16-byte aligned
        rows_total += n[m];
    }
    b->total_rows = rows_total;
    for (int64_t z : b->nnz) b->total_nnz += z;
    std::vector<int32_t> hptr((size_t)ptr_total);
    std::vector<int32_t> hcol((size_t)ent_total, 0);
    std::vector<double> hval((size_t)ent_total, 0.0);
    b->csr_items.assign(count, {});
    b->sliced_items.assign(count, {});
    b->csr_cost.assign(count, {});
    b->sliced_cost.assign(count, {});
    b->sliced_built.assign(count, 0);
    for (int m = 0; m < count; ++m) {
        const BatchMat& M = b->mats[m];
        const int64_t base = n[m] > 0 ? row_ptr[m][0] : 0;
        for (int64_t i = 0; i <= n[m]; ++i)
            hptr[(size_t)(M.ptr_off + i)] = n[m] > 0 ? (int32_t)(row_ptr[m][i] - base) : 0;
        for (int64_t k = 0; k < b->nnz[m]; ++k) {
            hcol[(size_t)(M.ent_off + k)] = col_idx[m][base + k];
            hval[(size_t)(M.ent_off + k)] = vals[m][base + k];
        }
        for (int64_t r = 0; r < n[m]; r += kItemRows) {
            const int64_t e = std::min<int64_t>(n[m], r + kItemRows);
            b->csr_items[m].push_back(BatchItem{m, 0, (int)r, (int)e});
            b->csr_cost[m].push_back((row_ptr[m][e] - row_ptr[m][r]) + 8 * (e - r));
        }
    }
    b->ptr = static_cast<int32_t*>(balloc(b, hptr.size() * 4));
    b->col = static_cast<int32_t*>(balloc(b, hcol.size() * 4));
    b->val = static_cast<double*>(balloc(b, hval.size() * 8));
    b->d_mats = static_cast<BatchMat*>(balloc(b, b->mats.size() * sizeof(BatchMat)));
    b->ticket = static_cast<int*>(balloc(b, 2 * sizeof(int)));
    spmvk::check_cuda(cudaMemcpy(b->ptr, hptr.data(), hptr.size() * 4, cudaMemcpyHostToDevice), "upload");
    spmvk::check_cuda(cudaMemcpy(b->col, hcol.data(), hcol.size() * 4, cudaMemcpyHostToDevice), "upload");
    spmvk::check_cuda(cudaMemcpy(b->val, hval.data(), hval.size() * 8, cudaMemcpyHostToDevice), "upload");
    spmvk::check_cuda(cudaMemcpy(b->d_mats, b->mats.data(), b->mats.size() * sizeof(BatchMat),
                                 cudaMemcpyHostToDevice), "upload");
    upload_items(b);
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
    for (cudaEvent_t ev : b->io_ev)
        if (ev) cudaEventDestroy(ev);
    bfree(b);
    delete b;
    return e == cudaSuccess ? SPMV_OK : bfail(SPMV_ECUDA, cudaGetErrorString(e));
}

int spmv_batch_set_lanes(spmv_batch* b, int m, int lanes) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    if (m < -1 || m >= b->count) spmvk::fail(SPMV_EINVAL, "matrix %d", m);
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32 &&
        lanes != kSliced)
        spmvk::fail(SPMV_EINVAL, "lanes %d not in {0,1,2,4,8,16,32,64}", lanes);
    spmvk::check_cuda(cudaDeviceSynchronize(), "synchronize");   // no launch may read the tables
    if (lanes != kSliced) batch_restore_csr(b);                    // the CSR modes read every row
    const int lo = m < 0 ? 0 : m, hi = m < 0 ? b->count : m + 1;
    bool changed = false;
    for (int i = lo; i < hi; ++i) {
        if (lanes == kSliced && !b->sliced_built[i]) build_sliced(b, i);
        changed = changed || ((b->mats[i].lanes == kSliced) != (lanes == kSliced));
        b->mats[i].lanes = lanes;
    }
    spmvk::check_cuda(cudaMemcpy(b->d_mats + lo, b->mats.data() + lo, (size_t)(hi - lo) * sizeof(BatchMat),
                                 cudaMemcpyHostToDevice),
                      "lanes");
    if (changed) upload_items(b);
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
        case SPMV_BQ_LAUNCHES:
            *out = (b->n_sliced_items > 0) + (b->n_items > b->n_sliced_items);
            break;
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
    spmvk::check_cuda(cudaMemsetAsync(b->ticket, 0, 2 * sizeof(int), s), "ticket reset");
    const int n_sl = b->n_sliced_items, n_csr = b->n_items - b->n_sliced_items;
    if (n_sl > 0) {
        BatchArgs a = args_of(b, x, y);
        a.order = b->d_order_full;
        a.n_items = n_sl;
        int grid = b->num_sms * std::max(1, b->occupancy_sliced);
        const int need = (n_sl + kThreads / 32 - 1) / (kThreads / 32);
        if (grid > need) grid = need;
        batch_sliced_persistent_kernel<<<grid, kThreads, 0, s>>>(a);
        spmvk::check_cuda(cudaGetLastError(), "batch launch (sliced)");
    }
    if (n_csr > 0) {
        BatchArgs a = args_of(b, x, y);
        a.order += n_sl;
        a.n_items = n_csr;
        a.ticket += 1;
        int grid = b->num_sms * std::max(1, b->occupancy);
        const int need = (n_csr + kThreads / 32 - 1) / (kThreads / 32);
        if (grid > need) grid = need;
        batch_persistent_kernel<<<grid, kThreads, 0, s>>>(a);
        spmvk::check_cuda(cudaGetLastError(), "batch launch");
    }
    BATCH_CATCH
    return SPMV_OK;
}

int spmv_batch_run_host(spmv_batch* b, const double* x_host, double* y_host, int chunks, cudaStream_t s_in,
                        cudaStream_t s_compute, cudaStream_t s_out) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    if (b->total_rows > 0 && (!x_host || !y_host)) spmvk::fail(SPMV_EINVAL, "host buffer is NULL");
    if (chunks < 1 || chunks > 64) spmvk::fail(SPMV_EINVAL, "chunks = %d not in [1, 64]", chunks);
    if (s_in == s_compute || s_out == s_compute || s_in == s_out) spmvk::fail(SPMV_EINVAL, "the streams must differ");
    if (b->total_rows == 0) return SPMV_OK;
    batch_host_setup(b);
    batch_host_product(b, x_host, y_host, b->io_x, b->io_y, chunks, s_in, s_compute, s_out, -1);
    spmvk::check_cuda(cudaStreamSynchronize(s_out), "synchronize");
    BATCH_CATCH
    return SPMV_OK;
}

int spmv_batch_run_host_many(spmv_batch* b, int64_t count, const double* x_host, int64_t x_stride, double* y_host,
                             int64_t y_stride, int chunks, cudaStream_t s_in, cudaStream_t s_compute,
                             cudaStream_t s_out) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    if (count < 0) spmvk::fail(SPMV_EINVAL, "count = %lld < 0", (long long)count);
    if (x_stride < 0 || y_stride < 0) spmvk::fail(SPMV_EINVAL, "negative stride");
    if (b->total_rows > 0 && count > 0 && (!x_host || !y_host)) spmvk::fail(SPMV_EINVAL, "host buffer is NULL");
    if (chunks < 1 || chunks > 64) spmvk::fail(SPMV_EINVAL, "chunks = %d not in [1, 64]", chunks);
    if (s_in == s_compute || s_out == s_compute || s_in == s_out) spmvk::fail(SPMV_EINVAL, "the streams must differ");
    if (count >= 2 && y_stride != 0 && y_stride < b->total_rows)
        spmvk::fail(SPMV_EINVAL, "y_stride %lld overlaps the results of consecutive products", (long long)y_stride);
    if (b->total_rows == 0 || count == 0) return SPMV_OK;
    batch_host_setup(b);
    if (!b->io_x2) {
        b->io_x2 = static_cast<double*>(balloc(b, (size_t)b->total_rows * sizeof(double)));
        b->io_y2 = static_cast<double*>(balloc(b, (size_t)b->total_rows * sizeof(double)));
    }
    for (int64_t k = 0; k < count; ++k) {
        const int slot = (int)(k & 1);
        batch_host_product(b, x_host + k * x_stride, y_host + k * y_stride, slot ? b->io_x2 : b->io_x,
                           slot ? b->io_y2 : b->io_y, chunks, s_in, s_compute, s_out, slot);
    }
    spmvk::check_cuda(cudaStreamSynchronize(s_out), "synchronize");
    spmvk::check_cuda(cudaStreamSynchronize(s_compute), "synchronize");
    spmvk::check_cuda(cudaStreamSynchronize(s_in), "synchronize");
    BATCH_CATCH
    return SPMV_OK;
}

int spmv_batch_release_csr(spmv_batch* b) {
    BATCH_TRY
    if (!b) spmvk::fail(SPMV_EINVAL, "batch is NULL");
    batch_release_csr(b);
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
        const bool sliced = b->mats[i].lanes == kSliced;
        int grid = b->num_sms * std::max(1, sliced ? b->occupancy_sliced : b->occupancy);
        const int need = (last - first + kThreads / 32 - 1) / (kThreads / 32);
        if (grid > need) grid = need;
        if (sliced)
            batch_sliced_range_kernel<<<grid, kThreads, 0, s>>>(a, first, last);
        else
            batch_range_kernel<<<grid, kThreads, 0, s>>>(a, first, last);
        spmvk::check_cuda(cudaGetLastError(), "matrix launch");
    }
    BATCH_CATCH
    return SPMV_OK;
}

}  // extern "C"
