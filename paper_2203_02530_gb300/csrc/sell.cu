// Sliced-ELL form of the CSR products y_L = A_L x_L and y += A_R x_R
// (Sec. III-A): the plan re-lays each rank's rows out in slices of 32
// positions, entry j of the slice's lane r at off + 32 j + r, every row
// padded to the slice's longest row (value 0, column 0).  A rank keeps its
// natural row order when that pads little; otherwise its rows are sorted by
// length, so a slice holds rows of similar length (a row permutation maps
// positions back to rows).  Rows longer than 64 entries are summed by whole
// warps instead.
//
// Why on GB300: FP64 FMA issues at 2 lanes per clock per SM, so the product
// is co-bound by HBM and the FP64 pipe and the cost that decides is warp
// DFMA instructions per entry.  In this layout one thread walks one row, so
// every stored entry costs exactly one lane-FMA with no shuffle reduction,
// and the 32 lanes of a warp read 32 consecutive values (256 bytes) and 32
// consecutive columns (128 bytes) per step: full coalescing without a
// shared-memory stage, so occupancy is set by registers alone.  On banded
// and stencil matrices the lanes' x gathers of one step are also contiguous
// rows of x.  Where every |column - row| of the LOCAL product fits 16 bits
// the columns can be kept as 16-bit deltas to the row instead (64 bytes per
// step), the 27-point stencil's case.  Each short row is summed in its CSR
// storage order, one FMA
// per entry from 0.0; padded slots are discarded by a select, so y equals
// that of the other one-thread-per-row kernels bit for bit.
#include "internal.h"
#include "pdl.cuh"

#include <cuda_runtime.h>

namespace spmvk {

namespace {

__device__ __forceinline__ uint64_t sell_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t sell_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Streamed operand, read once: skip L1, evict first from L2.
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int16_t* p, uint64_t pol) {
    int32_t v;   // sign-extended
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s16 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// Gathered x, reused across rows: keep in L2.
__device__ __forceinline__ double ld_keep(const double* p, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void sell_store(const CsrArgs& a, int row, double sum) {
    if (a.rowmap) {
        const int o = __ldg(a.rowmap + row);
        a.y[o] = a.accumulate ? a.y[o] + sum : sum;
    } else {
        a.y[row] = a.accumulate ? a.y[row] + sum : sum;
    }
}

// K consecutive slots j .. j + K - 1 of a slice lane: K value and K column
// loads, then K x gathers, then K FMAs in slot order (slots at or past the
// lane's row length discarded by a select).
template <int K, typename CT>
__device__ __forceinline__ void sell_round(const CT* cp, const double* vp, const double* xb, int j, int len,
                                           double& sum, uint64_t pol_stream, uint64_t pol_keep) {
    int32_t c[K];
    double v[K], xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        c[u] = ld_stream(cp + 32 * (j + u), pol_stream);
        v[u] = ld_stream(vp + 32 * (j + u), pol_stream);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) xv[u] = ld_keep(xb + c[u], pol_keep);
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const double t = fma(v[u], xv[u], sum);
        sum = (j + u < len) ? t : sum;
    }
}

// The r < U remaining slots of a slice lane as one round of r.
template <int U, typename CT>
__device__ __forceinline__ void sell_tail(int r, const CT* cp, const double* vp, const double* xb, int j, int len,
                                          double& sum, uint64_t pol_stream, uint64_t pol_keep) {
    switch (r) {
        case 1: sell_round<1>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 2: if (U > 2) sell_round<2>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 3: if (U > 3) sell_round<3>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 4: if (U > 4) sell_round<4>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 5: if (U > 5) sell_round<5>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 6: if (U > 6) sell_round<6>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 7: if (U > 7) sell_round<7>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        case 8: if (U > 8) sell_round<8>(cp, vp, xb, j, len, sum, pol_stream, pol_keep); break;
        default: break;
    }
}

// Entries [k, ke) of a long row taken by one lane in steps of 32 (k = the
// lane's first), R at a time: R value and R column loads, then R gathers,
// then R FMAs in entry order; in the last round the entries at or past ke
// are neither loaded nor added.
template <int R>
__device__ __forceinline__ void long_round(const CsrArgs& a, const double* xb, int k, int ke, double& part,
                                           uint64_t pol_stream, uint64_t pol_keep) {
    double v[R], xv[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const bool m = k + 32 * u < ke;
        v[u] = m ? ld_stream(a.val + k + 32 * u, pol_stream) : 0.0;
        const int c = m ? ld_stream(a.col + k + 32 * u, pol_stream) : 0;
        xv[u] = m ? ld_keep(xb + c, pol_keep) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const double t = fma(v[u], xv[u], part);
        part = k + 32 * u < ke ? t : part;
    }
}

}  // namespace

// One warp per work unit, grid-stride: units [0, n_long) are the launch's
// long rows (each summed by the whole warp: lane l takes entries l, l+32,
// ... in order, then a fixed xor-butterfly), the rest its slices (one lane
// per row, U entries per lane per step: U value and U column loads, then U
// x gathers, then U FMAs, so each lane keeps U gathers in flight; the slots
// past the last full step go in rounds of 4, 2 and 1, the long rows' last
// entries in a round of 2 and 1).  Long rows come first so that the
// heaviest units start in the first wave.
// With sa.cta_off the units are split into contiguous cost-balanced ranges
// instead, one per CTA, whose 8 warps take the range round-robin.
// CT = int32_t: slot columns are the CSR's (x index = xoff + column);
// CT = int16_t: slot columns are deltas to the row (x index = row + delta),
// half the index bytes where every |column - row| fits in 16 bits.
// YP: the layout has a y row per position (sa.ypos; sorted remote layouts).
template <int U, int MINB, typename CT, bool YP = false>
__global__ void __launch_bounds__(256, MINB) csr_sell_kernel(CsrArgs a, SellArgs sa) {
    // the previous kernel of this stream is done (unless independent, or
    // the wait is deferred to the first access to y)
    pdl_begin_deferrable(a.pdl);
    bool pending = (a.pdl & kPdlDefer) != 0;
    constexpr bool kDelta = sizeof(CT) == 2;
    const uint64_t pol_stream = sell_policy_evict_first();
    const uint64_t pol_keep = sell_policy_evict_last();
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * 8;
    const int n_long = sa.long_end - sa.long_begin;
    const int n_units = n_long + (sa.slice_end - sa.slice_begin);
    int u0 = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5), u_end = n_units, stride = nwarps;
    if (sa.cta_off) {
        u0 = __ldg(sa.cta_off + blockIdx.x) + (int)(threadIdx.x >> 5);
        u_end = __ldg(sa.cta_off + blockIdx.x + 1);
        stride = 8;
    }
    for (; u0 < u_end; u0 += stride) {
        if (u0 < n_long) {
            const SellLong L = sa.longs[sa.long_begin + u0];
            const int kb = L.k0, ke = L.k1;
            const double* xb = a.x + L.xoff;
            double part = 0.0;
            if (U >= 8) {
                // the lane's entries kb + lane, + 32, ... in rounds of 8 (at
                // most 16 per lane: a piece holds at most 512 entries); the
                // last round is predicated per entry
                for (int k = kb + lane; k < ke; k += 256) long_round<8>(a, xb, k, ke, part, pol_stream, pol_keep);
            } else {
                // fewer registers: rounds of 4, then the lane's last 2 and 1
                int k = kb + lane;
                for (; k + 96 < ke; k += 128) {
                    double v[4], xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        v[u] = ld_stream(a.val + k + 32 * u, pol_stream);
                        xv[u] = ld_keep(xb + ld_stream(a.col + k + 32 * u, pol_stream), pol_keep);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) part = fma(v[u], xv[u], part);
                }
                if (k + 32 < ke) {
                    const double v0 = ld_stream(a.val + k, pol_stream), v1 = ld_stream(a.val + k + 32, pol_stream);
                    const int c0 = ld_stream(a.col + k, pol_stream), c1 = ld_stream(a.col + k + 32, pol_stream);
                    const double x0 = ld_keep(xb + c0, pol_keep), x1 = ld_keep(xb + c1, pol_keep);
                    part = fma(v0, x0, part);
                    part = fma(v1, x1, part);
                    k += 64;
                }
                if (k < ke)
                    part = fma(ld_stream(a.val + k, pol_stream),
                               ld_keep(xb + ld_stream(a.col + k, pol_stream), pol_keep), part);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            pdl_settle(pending);
            if (lane == 0) {
                if (L.nparts == 1) {
                    sell_store(a, L.row, part);
                } else {
                    // publish this piece, then the warp that completes the row
                    // adds its pieces in piece order (independent of timing)
                    sa.long_part[L.slot] = part;
                    __threadfence();
                    if (atomicAdd(sa.long_cnt + L.cidx, 1) == L.nparts - 1) {
                        __threadfence();
                        double sum = 0.0;
                        for (int i = 0; i < L.nparts; ++i) sum += __ldcg(sa.long_part + L.first + i);
                        sell_store(a, L.row, sum);
                        sa.long_cnt[L.cidx] = 0;   // ready for the next launch
                    }
                }
            }
            continue;
        }
        const SellSlice d = sa.slices[sa.slice_begin + u0 - n_long];
        const int pos = d.p0 + lane;
        int len = 0;
        bool store = false;
        if (lane < d.rows) {
            const int code = sa.len[pos];
            store = code != kSellLenLong;
            len = store ? code : 0;
        }
        const double* vp = sa.val + (int64_t)d.off + lane;
        const CT* cp = (kDelta ? reinterpret_cast<const CT*>(sa.col16) : reinterpret_cast<const CT*>(sa.col)) +
                       (int64_t)d.off + lane;
        int row = lane < d.rows ? pos : d.p0;   // lanes past the slice's rows gather x[p0] (padding)
        // with YP, `row` is the y row itself (row order and row map
        // composed), loaded here so that its latency hides behind the rounds
        if (YP) {
            if (lane < d.rows) row = __ldg(sa.ypos + pos);
        } else if (sa.perm && lane < d.rows) {
            row = __ldg(sa.perm + pos);
        }
        const double* xb = kDelta ? a.x + row : a.x + d.xoff;
        double sum = 0.0;
        int j = 0;
        for (; j + U <= d.len; j += U) sell_round<U>(cp, vp, xb, j, len, sum, pol_stream, pol_keep);
        // the last d.len mod U slots in one round of exactly that many (the
        // count is the same for the whole warp): one load-then-gather
        // latency, so the short slices of skewed rows (3 entries, say) keep
        // all their gathers in flight at once
        sell_tail<U>(d.len - j, cp, vp, xb, j, len, sum, pol_stream, pol_keep);
        pdl_settle(pending);
        if (store) {
            if (YP) a.y[row] = a.accumulate ? a.y[row] + sum : sum;
            else sell_store(a, row, sum);
        }
    }
    pdl_settle(pending);
}

// Fill the sliced arrays from the CSR: one warp per slice, one lane per
// position (a long row's slots, if it sits in a slice, stay padding).
__global__ void __launch_bounds__(256) sell_fill_kernel(const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const SellSlice* __restrict__ slices, int n_slices,
                                                        const uint8_t* __restrict__ lens,
                                                        const int32_t* __restrict__ perm,
                                                        double* __restrict__ sval, int32_t* __restrict__ scol) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * 8;
    for (int si = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); si < n_slices; si += nwarps) {
        const SellSlice d = slices[si];
        const int pos = d.p0 + lane;
        const bool live = lane < d.rows && lens[pos] != kSellLenLong;
        const int row = live ? (perm ? perm[pos] : pos) : 0;
        const int kb = live ? ptr[row] : 0;
        const int len = live ? ptr[row + 1] - kb : 0;
        for (int j = 0; j < d.len; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            sval[o] = j < len ? val[kb + j] : 0.0;
            scol[o] = j < len ? col[kb + j] : 0;
        }
    }
}

// 16-bit column deltas of a filled layout: slot (slice, j, lane) gets
// xoff + column - row of its row, padding 0; *bad is set when a delta does
// not fit (the 16-bit copy is then unusable).
__global__ void __launch_bounds__(256) sell_delta_kernel(const SellSlice* __restrict__ slices, int n_slices,
                                                         const uint8_t* __restrict__ lens,
                                                         const int32_t* __restrict__ perm,
                                                         const int32_t* __restrict__ scol,
                                                         int16_t* __restrict__ scol16, int* bad) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * 8;
    for (int si = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); si < n_slices; si += nwarps) {
        const SellSlice d = slices[si];
        const int pos = d.p0 + lane;
        const bool live = lane < d.rows && lens[pos] != kSellLenLong;
        const int len = live ? lens[pos] : 0;
        const int row = live ? (perm ? perm[pos] : pos) : 0;
        for (int j = 0; j < d.len; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            int delta = 0;
            if (j < len) {
                delta = d.xoff + scol[o] - row;
                if (delta < -32768 || delta > 32767) {
                    atomicOr(bad, 1);
                    delta = 0;
                }
            }
            scol16[o] = (int16_t)delta;
        }
    }
}

cudaError_t launch_sell_delta(const SellSlice* slices, int n_slices, const uint8_t* len, const int32_t* perm,
                              const int32_t* scol, int16_t* scol16, int* bad, int num_sms, cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    int grid = (n_slices + 7) / 8;
    if (grid > num_sms * 8) grid = num_sms * 8;
    sell_delta_kernel<<<grid, 256, 0, s>>>(slices, n_slices, len, perm, scol, scol16, bad);
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(const int32_t* ptr, const int32_t* col, const double* val, const SellSlice* slices,
                             int n_slices, const uint8_t* len, const int32_t* perm, double* sval, int32_t* scol,
                             int num_sms, cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    int grid = (n_slices + 7) / 8;
    if (grid > num_sms * 8) grid = num_sms * 8;
    sell_fill_kernel<<<grid, 256, 0, s>>>(ptr, col, val, slices, n_slices, len, perm, sval, scol);
    return cudaGetLastError();
}

// Moves of index ranges: segment s (one warp) copies len values and columns
// from position src of (sv, sc) to position dst of (dv, dc); tab holds
// (src, dst, len) per segment.  Used to move long rows between the CSR and
// the compact long-row arrays of a plan whose CSR is released.
__global__ void __launch_bounds__(256) segment_copy_kernel(const int32_t* __restrict__ tab, int n_seg,
                                                           const double* __restrict__ sv,
                                                           const int32_t* __restrict__ sc, double* __restrict__ dv,
                                                           int32_t* __restrict__ dc) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * 8;
    for (int g = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); g < n_seg; g += nwarps) {
        const int src = __ldg(tab + 3 * g), dst = __ldg(tab + 3 * g + 1), len = __ldg(tab + 3 * g + 2);
        for (int i = lane; i < len; i += 32) {
            dv[dst + i] = sv[src + i];
            dc[dst + i] = sc[src + i];
        }
    }
}

// The inverse of sell_fill_kernel: the live slots of every slice back into
// their CSR rows (ptr of the CSR the layout was filled from).  Columns come
// from the 32-bit slots, or, when scol is null, from the 16-bit deltas
// (column = row + delta - xoff, the inverse of sell_delta_kernel).
__global__ void __launch_bounds__(256) sell_unfill_kernel(const int32_t* __restrict__ ptr,
                                                          const SellSlice* __restrict__ slices, int n_slices,
                                                          const uint8_t* __restrict__ lens,
                                                          const int32_t* __restrict__ perm,
                                                          const double* __restrict__ sval,
                                                          const int32_t* __restrict__ scol,
                                                          const int16_t* __restrict__ scol16,
                                                          int32_t* __restrict__ col, double* __restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * 8;
    for (int si = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); si < n_slices; si += nwarps) {
        const SellSlice d = slices[si];
        const int pos = d.p0 + lane;
        const bool live = lane < d.rows && lens[pos] != kSellLenLong;
        const int row = live ? (perm ? perm[pos] : pos) : 0;
        const int kb = live ? ptr[row] : 0;
        const int len = live ? lens[pos] : 0;
        for (int j = 0; j < len; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            val[kb + j] = sval[o];
            col[kb + j] = scol ? scol[o] : row + (int)scol16[o] - d.xoff;
        }
    }
}

// 32-bit slot columns of a layout from its 16-bit deltas (padding 0, as
// sell_fill_kernel writes it).
__global__ void __launch_bounds__(256) sell_col32_kernel(const SellSlice* __restrict__ slices, int n_slices,
                                                         const uint8_t* __restrict__ lens,
                                                         const int32_t* __restrict__ perm,
                                                         const int16_t* __restrict__ scol16,
                                                         int32_t* __restrict__ scol) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)gridDim.x * 8;
    for (int si = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5); si < n_slices; si += nwarps) {
        const SellSlice d = slices[si];
        const int pos = d.p0 + lane;
        const bool live = lane < d.rows && lens[pos] != kSellLenLong;
        const int row = live ? (perm ? perm[pos] : pos) : 0;
        const int len = live ? lens[pos] : 0;
        for (int j = 0; j < d.len; ++j) {
            const int64_t o = (int64_t)d.off + 32 * j + lane;
            scol[o] = j < len ? row + (int)scol16[o] - d.xoff : 0;
        }
    }
}

static int warp_grid(int items, int num_sms) {
    int grid = (items + 7) / 8;
    if (grid > num_sms * 8) grid = num_sms * 8;
    return grid;
}

cudaError_t launch_segment_copy(const int32_t* tab, int n_seg, const double* sv, const int32_t* sc, double* dv,
                                int32_t* dc, int num_sms, cudaStream_t s) {
    if (n_seg <= 0) return cudaSuccess;
    segment_copy_kernel<<<warp_grid(n_seg, num_sms), 256, 0, s>>>(tab, n_seg, sv, sc, dv, dc);
    return cudaGetLastError();
}

cudaError_t launch_sell_unfill(const int32_t* ptr, const SellSlice* slices, int n_slices, const uint8_t* len,
                               const int32_t* perm, const double* sval, const int32_t* scol, const int16_t* scol16,
                               int32_t* col, double* val, int num_sms, cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    sell_unfill_kernel<<<warp_grid(n_slices, num_sms), 256, 0, s>>>(ptr, slices, n_slices, len, perm, sval, scol,
                                                                    scol16, col, val);
    return cudaGetLastError();
}

cudaError_t launch_sell_col32(const SellSlice* slices, int n_slices, const uint8_t* len, const int32_t* perm,
                              const int16_t* scol16, int32_t* scol, int num_sms, cudaStream_t s) {
    if (n_slices <= 0) return cudaSuccess;
    sell_col32_kernel<<<warp_grid(n_slices, num_sms), 256, 0, s>>>(slices, n_slices, len, perm, scol16, scol);
    return cudaGetLastError();
}

bool sell_param_supported(int param) {
    const int base = param >= 2000 ? param - 2000 : param;
    return base == 4 || base == 8 || base == 9 || (base >= 104 && base <= 107);
}

int sell_grid(int param, int units, int num_sms) {
    int blocks_per_sm = 0;
    switch (param % 1000) {
        case 4: blocks_per_sm = 8; break;
        case 8: blocks_per_sm = 4; break;
        case 9: blocks_per_sm = 4; break;
        case 104: blocks_per_sm = 6; break;
        case 105: blocks_per_sm = 5; break;
        case 106: blocks_per_sm = 6; break;
        case 107: blocks_per_sm = 5; break;
        default: return 0;
    }
    if (units <= 0) return 0;
    int grid = num_sms * blocks_per_sm;
    if (grid > (units + 7) / 8) grid = (units + 7) / 8;
    return grid;
}

cudaError_t launch_sell(const CsrArgs& a, const SellArgs& sa, int param, bool delta16, int num_sms,
                        cudaStream_t st) {
    const int units = (sa.long_end - sa.long_begin) + (sa.slice_end - sa.slice_begin);
    if (units <= 0) return cudaSuccess;
    const int grid = sell_grid(param, units, num_sms);
    if (grid <= 0) return cudaErrorInvalidValue;
    if (sell_param_balanced(param) != (sa.cta_off != nullptr)) return cudaErrorInvalidValue;
#define SELL_LAUNCH(u, b)                                                                        \
    e = delta16 ? launch_pdl(csr_sell_kernel<u, b, int16_t>, dim3(grid), dim3(256), 0, st, a, sa)      \
        : sa.ypos ? launch_pdl(csr_sell_kernel<u, b, int32_t, true>, dim3(grid), dim3(256), 0, st, a, sa) \
                  : launch_pdl(csr_sell_kernel<u, b, int32_t>, dim3(grid), dim3(256), 0, st, a, sa)
    cudaError_t e = cudaSuccess;
    switch (param % 1000) {
        case 4: SELL_LAUNCH(4, 8); break;
        case 8: SELL_LAUNCH(8, 4); break;
        case 9: SELL_LAUNCH(9, 4); break;
        case 104: SELL_LAUNCH(4, 6); break;
        case 105: SELL_LAUNCH(8, 5); break;
        case 106: SELL_LAUNCH(8, 6); break;
        case 107: SELL_LAUNCH(9, 5); break;
        default: return cudaErrorInvalidValue;
    }
#undef SELL_LAUNCH
    return e;
}

}  // namespace spmvk
