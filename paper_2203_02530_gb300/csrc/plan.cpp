// Partition plan of the row-partitioned SpMV (Sec. III-A, Fig. 3b of
// Pearson, Javeed and Devine), built on the host once and kept in HBM:
//   - P contiguous, even row blocks r_p = floor(p n / P);
//   - A_L: the entries of block p whose column lies in the block, columns
//     rebased so that x_L = x + r_p ("A_L x_L can be computed directly");
//   - H_p: the distinct remote columns of block p, ascending ("A is static,
//     so the entries that make up x_R are fixed");
//   - A_R: the remaining entries, columns renumbered to positions in the
//     receive buffer (the column-compressed off-diagonal block), stored only
//     for rows that have remote entries;
//   - send buffer slots destination-major, then source rank, then ascending
//     column, so destination p's part is x[H_p] and the exchange is one copy.
#include "part.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

namespace spmvk {

constexpr int64_t kBlockRows = 256;

void fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    throw Fail{code, std::string(buf)};
}

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    cudaGetLastError();   // clear a non-sticky error
    if (e == cudaErrorMemoryAllocation) fail(SPMV_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    fail(SPMV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* dev_alloc(spmv_part* pt, size_t bytes) {
    void* p = nullptr;
    const size_t total = bytes + kPad;
    check_cuda(cudaMalloc(&p, total), "cudaMalloc");
    pt->allocs.push_back(DevArray{p, bytes});
    pt->device_bytes += total;
    cudaError_t e = cudaMemset(p, 0, total);
    check_cuda(e, "cudaMemset");
    return p;
}

template <class T>
static T* upload(spmv_part* pt, const std::vector<T>& h) {
    T* d = static_cast<T*>(dev_alloc(pt, h.size() * sizeof(T)));
    if (!h.empty())
        check_cuda(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice),
                   "upload");
    return d;
}

static void free_one(spmv_part* pt, void* p) {
    if (!p) return;
    for (size_t i = 0; i < pt->allocs.size(); ++i) {
        if (pt->allocs[i].p == p) {
            cudaFree(p);
            pt->device_bytes -= pt->allocs[i].bytes + kPad;
            pt->allocs.erase(pt->allocs.begin() + (long)i);
            return;
        }
    }
}

void free_plan(spmv_part* pt) {
    for (auto& g : pt->graphs)
        if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
    pt->graphs.clear();
    for (cudaEvent_t e : pt->op_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : pt->join_ev)
        if (e) cudaEventDestroy(e);
    if (pt->fork_ev) cudaEventDestroy(pt->fork_ev);
    for (cudaEvent_t e : pt->io_ev)
        if (e) cudaEventDestroy(e);
    pt->io_ev.clear();
    if (pt->io_out) cudaStreamDestroy(pt->io_out);
    if (pt->io_alt) cudaStreamDestroy(pt->io_alt);
    if (pt->io_aux) cudaStreamDestroy(pt->io_aux);
    pt->io_out = nullptr;
    pt->io_alt = nullptr;
    pt->io_aux = nullptr;
    pt->op_ev.clear();
    pt->join_ev.clear();
    pt->fork_ev = nullptr;
    for (auto& a : pt->allocs) cudaFree(a.p);
    pt->allocs.clear();
    pt->device_bytes = 0;
}

void validate_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, int P) {
    if (n < 0) fail(SPMV_EINVAL, "n = %lld < 0", (long long)n);
    if (n >= (int64_t(1) << 31)) fail(SPMV_EBOUNDS, "n = %lld needs 64-bit columns", (long long)n);
    if (P < 1) fail(SPMV_EINVAL, "P = %d < 1", P);
    if (P > 1024) fail(SPMV_EBOUNDS, "P = %d above the limit 1024", P);
    if (!rp) fail(SPMV_EINVAL, "row_ptr is NULL");
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) fail(SPMV_EINVAL, "row_ptr decreases at row %lld", (long long)i);
    const int64_t nnz = rp[n] - rp[0];
    if (nnz >= (int64_t(1) << 31) - 64) fail(SPMV_EBOUNDS, "nnz = %lld too large", (long long)nnz);
    if (nnz > 0 && (!ci || !va)) fail(SPMV_EINVAL, "col_idx or vals is NULL");
    for (int64_t k = rp[0]; k < rp[n]; ++k)
        if (ci[k] < 0 || ci[k] >= n)
            fail(SPMV_EINVAL, "column %d out of range at entry %lld", ci[k], (long long)(k - rp[0]));
}

void build_plan(spmv_part* pt, int64_t n, const int64_t* rp, const int32_t* ci,
                const double* va) {
    const int P = pt->P;
    validate_csr(n, rp, ci, va, P);
    if (n < 0) fail(SPMV_EINVAL, "n = %lld < 0", (long long)n);
    if (n >= (int64_t(1) << 31)) fail(SPMV_EBOUNDS, "n = %lld needs 64-bit columns", (long long)n);
    if (P < 1) fail(SPMV_EINVAL, "P = %d < 1", P);
    if (P > 1024) fail(SPMV_EBOUNDS, "P = %d above the limit 1024", P);
    if (!rp) fail(SPMV_EINVAL, "row_ptr is NULL");
    const int64_t base = rp[0];
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) fail(SPMV_EINVAL, "row_ptr decreases at row %lld", (long long)i);
    const int64_t nnz = rp[n] - base;
    if (nnz >= (int64_t(1) << 31) - 64) fail(SPMV_EBOUNDS, "nnz = %lld too large", (long long)nnz);
    if (nnz > 0 && (!ci || !va)) fail(SPMV_EINVAL, "col_idx or vals is NULL");
    for (int64_t k = base; k < rp[n]; ++k)
        if (ci[k] < 0 || ci[k] >= n)
            fail(SPMV_EINVAL, "column %d out of range at entry %lld", ci[k], (long long)(k - base));

    pt->n = n;
    pt->nnz = nnz;
    pt->bounds.resize(P + 1);
    for (int p = 0; p <= P; ++p) pt->bounds[p] = (int64_t)p * n / P;
    const std::vector<int64_t>& B = pt->bounds;

    // ---- split rows into A_L (global row order) and A_R (compressed rows)
    std::vector<int32_t> l_ptr(n + 1, 0), l_col;
    std::vector<double> l_val;
    std::vector<int32_t> rr_row, rr_ptr(1, 0), r_col;
    std::vector<double> r_val;
    int64_t n_local = 0;
    l_col.reserve((size_t)nnz);
    l_val.reserve((size_t)nnz);
    pt->rr_off.assign(P + 1, 0);
    pt->halo_off.assign(P + 1, 0);
    std::vector<int32_t> send_idx;
    std::vector<int32_t> stamp(n > 0 ? (size_t)n : 1, -1), pos(n > 0 ? (size_t)n : 1, 0);
    std::vector<int32_t> distinct;
    for (int p = 0; p < P; ++p) {
        const int64_t rb = B[p], re = B[p + 1];
        pt->rr_off[p] = (int64_t)rr_row.size();
        const size_t r_first = r_col.size();
        for (int64_t i = rb; i < re; ++i) {
            int32_t nr = 0;
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t c = ci[k];
                if (c >= rb && c < re) {
                    l_col.push_back((int32_t)(c - rb));
                    l_val.push_back(va[k]);
                    ++n_local;
                } else {
                    r_col.push_back(c);   // global column for now
                    r_val.push_back(va[k]);
                    if (stamp[(size_t)c] != p) {
                        stamp[(size_t)c] = p;
                        distinct.push_back(c);
                    }
                    ++nr;
                }
            }
            l_ptr[(size_t)i + 1] = (int32_t)n_local;
            if (nr) {
                rr_row.push_back((int32_t)i);
                rr_ptr.push_back((int32_t)r_col.size());
            }
        }
        // H_p: the distinct remote columns, ascending; a column's slot in
        // the receive buffer is halo_off[p] + its rank in H_p
        pt->halo_off[p] = (int64_t)send_idx.size();
        std::sort(distinct.begin(), distinct.end());
        for (int32_t c : distinct) {
            pos[(size_t)c] = (int32_t)send_idx.size();
            send_idx.push_back(c);
        }
        distinct.clear();
        for (size_t k = r_first; k < r_col.size(); ++k) r_col[k] = pos[(size_t)r_col[k]];
    }
    pt->rr_off[P] = (int64_t)rr_row.size();
    pt->halo_off[P] = (int64_t)send_idx.size();
    pt->nnz_l = n_local;
    pt->nnz_r = (int64_t)r_col.size();
    pt->n_send = (int64_t)send_idx.size();
    pt->n_rr = (int64_t)rr_row.size();

    // ---- segments (dst p, src q): H_p is ascending and q's columns are a
    // contiguous range, so each segment is a contiguous slice of p's part
    pt->seg_off.assign((size_t)P * P + 1, 0);
    for (int p = 0; p < P; ++p) {
        const int32_t* h0 = send_idx.data() + pt->halo_off[p];
        const int32_t* h1 = send_idx.data() + pt->halo_off[p + 1];
        for (int q = 0; q < P; ++q) {
            const int32_t* at = std::lower_bound(h0, h1, (int32_t)B[q]);
            pt->seg_off[(size_t)p * P + q] = pt->halo_off[p] + (at - h0);
        }
    }
    pt->seg_off[(size_t)P * P] = pt->n_send;

    // ---- send slots grouped by source rank (per-rank Pack ops)
    std::vector<int32_t> pack_pos;
    pack_pos.reserve((size_t)pt->n_send);
    pt->pack_off.assign(P + 1, 0);
    for (int q = 0; q < P; ++q) {
        pt->pack_off[q] = (int64_t)pack_pos.size();
        for (int p = 0; p < P; ++p) {
            const int64_t s0 = pt->seg_off[(size_t)p * P + q];
            const int64_t s1 = pt->seg_off[(size_t)p * P + q + 1];
            for (int64_t k = s0; k < s1; ++k) pack_pos.push_back((int32_t)k);
        }
    }
    pt->pack_off[P] = (int64_t)pack_pos.size();

    // ---- upload
    pt->l_ptr = upload(pt, l_ptr);
    pt->l_col = upload(pt, l_col);
    pt->l_val = upload(pt, l_val);
    pt->rr_row = upload(pt, rr_row);
    pt->rr_ptr = upload(pt, rr_ptr);
    pt->r_col = upload(pt, r_col);
    pt->r_val = upload(pt, r_val);
    pt->send_idx = upload(pt, send_idx);
    pt->pack_pos = upload(pt, pack_pos);
    pt->sendbuf = static_cast<double*>(dev_alloc(pt, (size_t)pt->n_send * sizeof(double)));
    pt->recvbuf = static_cast<double*>(dev_alloc(pt, (size_t)pt->n_send * sizeof(double)));
    pt->err = static_cast<int*>(dev_alloc(pt, sizeof(int)));
}

// Greedy row tiles of one CSR row range: consecutive rows while the tile
// holds at most g.rows() rows and g.nnz_cap entries; a row longer than the
// capacity gets a tile of its own marked TILE_LONG.
static void tile_range(const std::vector<int32_t>& ptr, int64_t rb, int64_t re, int32_t xoff,
                       const TileGeom& g, std::vector<Tile>& out) {
    int64_t r = rb;
    while (r < re) {
        const int64_t len = (int64_t)ptr[(size_t)r + 1] - ptr[(size_t)r];
        if (len > g.nnz_cap) {
            out.push_back(Tile{(int32_t)r, (int32_t)(r + 1), ptr[(size_t)r], ptr[(size_t)r + 1], xoff,
                               TILE_LONG, 0, 0});
            ++r;
            continue;
        }
        const int64_t start = r;
        int64_t cnt = 0;
        while (r < re && r - start < g.rows()) {
            const int64_t l = (int64_t)ptr[(size_t)r + 1] - ptr[(size_t)r];
            if (l > g.nnz_cap || cnt + l > g.nnz_cap) break;
            cnt += l;
            ++r;
        }
        out.push_back(Tile{(int32_t)start, (int32_t)r, ptr[(size_t)start], ptr[(size_t)r], xoff, 0, 0, 0});
    }
}

template <class T>
static std::vector<T> download(const T* d, size_t count) {
    std::vector<T> h(count);
    if (count) check_cuda(cudaMemcpy(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost), "download");
    return h;
}

void build_tiles(spmv_part* pt, const TileGeom& g) {
    const int P = pt->P;
    const std::vector<int32_t> l_ptr = download(pt->l_ptr, (size_t)pt->n + 1);
    const std::vector<int32_t> rr_ptr = download(pt->rr_ptr, (size_t)pt->n_rr + 1);
    std::vector<Tile> lt, rt;
    pt->ltile_off.assign(P + 1, 0);
    pt->rtile_off.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        pt->ltile_off[p] = (int64_t)lt.size();
        tile_range(l_ptr, pt->bounds[p], pt->bounds[p + 1], (int32_t)pt->bounds[p], g, lt);
        pt->rtile_off[p] = (int64_t)rt.size();
        tile_range(rr_ptr, pt->rr_off[p], pt->rr_off[p + 1], 0, g, rt);
    }
    pt->ltile_off[P] = (int64_t)lt.size();
    pt->rtile_off[P] = (int64_t)rt.size();
    free_one(pt, pt->ltiles);
    free_one(pt, pt->rtiles);
    pt->ltiles = upload(pt, lt);
    pt->rtiles = upload(pt, rt);
    pt->geom = g;
    if (!pt->lblocks) {
        std::vector<Tile> lb, rb;
        pt->lblock_off.assign(P + 1, 0);
        pt->rblock_off.assign(P + 1, 0);
        auto blocks = [](const std::vector<int32_t>& ptr, int64_t r0, int64_t r1, int32_t xoff,
                         std::vector<Tile>& out) {
            for (int64_t r = r0; r < r1; r += kBlockRows) {
                const int64_t e = std::min(r1, r + kBlockRows);
                out.push_back(Tile{(int32_t)r, (int32_t)e, ptr[(size_t)r], ptr[(size_t)e], xoff, 0, 0, 0});
            }
        };
        for (int p = 0; p < P; ++p) {
            pt->lblock_off[p] = (int64_t)lb.size();
            blocks(l_ptr, pt->bounds[p], pt->bounds[p + 1], (int32_t)pt->bounds[p], lb);
            pt->rblock_off[p] = (int64_t)rb.size();
            blocks(rr_ptr, pt->rr_off[p], pt->rr_off[p + 1], 0, rb);
        }
        pt->lblock_off[P] = (int64_t)lb.size();
        pt->rblock_off[P] = (int64_t)rb.size();
        pt->lblocks = upload(pt, lb);
        pt->rblocks = upload(pt, rb);
    }
}

// Merge-path tiles of every rank, local and remote, plus one carry slot
// per tile.  Coordinates come from a device-side path search on the row
// pointers the kernels use.
void build_merge_tiles(spmv_part* pt) {
    const int P = pt->P;
    const int items = merge_items_per_tile();
    std::vector<int32_t> l_ptr_b(P + 1), rr_ptr_b(P + 1);
    for (int p = 0; p <= P; ++p) {
        check_cuda(cudaMemcpy(&l_ptr_b[p], pt->l_ptr + pt->bounds[p], 4, cudaMemcpyDeviceToHost), "merge plan");
        check_cuda(cudaMemcpy(&rr_ptr_b[p], pt->rr_ptr + pt->rr_off[p], 4, cudaMemcpyDeviceToHost), "merge plan");
    }
    pt->lmtile_off.assign(P + 1, 0);
    pt->rmtile_off.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        const int64_t li = (pt->bounds[p + 1] - pt->bounds[p]) + (int64_t)(l_ptr_b[p + 1] - l_ptr_b[p]);
        const int64_t ri = (pt->rr_off[p + 1] - pt->rr_off[p]) + (int64_t)(rr_ptr_b[p + 1] - rr_ptr_b[p]);
        pt->lmtile_off[p + 1] = pt->lmtile_off[p] + (li + items - 1) / items;
        pt->rmtile_off[p + 1] = pt->rmtile_off[p] + (ri + items - 1) / items;
    }
    free_one(pt, pt->lmtiles);
    free_one(pt, pt->rmtiles);
    free_one(pt, pt->lcarry);
    free_one(pt, pt->rcarry);
    pt->lmtiles = static_cast<MergeTile*>(dev_alloc(pt, (size_t)pt->lmtile_off[P] * sizeof(MergeTile)));
    pt->rmtiles = static_cast<MergeTile*>(dev_alloc(pt, (size_t)pt->rmtile_off[P] * sizeof(MergeTile)));
    pt->lcarry = static_cast<Carry*>(dev_alloc(pt, (size_t)pt->lmtile_off[P] * sizeof(Carry)));
    pt->rcarry = static_cast<Carry*>(dev_alloc(pt, (size_t)pt->rmtile_off[P] * sizeof(Carry)));
    for (int p = 0; p < P; ++p) {
        check_cuda(launch_merge_partition(pt->l_ptr, (int)pt->bounds[p], (int)pt->bounds[p + 1],
                                          (int32_t)pt->bounds[p], pt->lmtiles + pt->lmtile_off[p],
                                          (int)(pt->lmtile_off[p + 1] - pt->lmtile_off[p]), 0),
                   "merge partition");
        check_cuda(launch_merge_partition(pt->rr_ptr, (int)pt->rr_off[p], (int)pt->rr_off[p + 1], 0,
                                          pt->rmtiles + pt->rmtile_off[p],
                                          (int)(pt->rmtile_off[p + 1] - pt->rmtile_off[p]), 0),
                   "merge partition");
    }
    check_cuda(cudaDeviceSynchronize(), "merge partition");
}

// Tiles of at most 32 rows and `cap` entries (one warp each).
void build_warp_tiles(spmv_part* pt, int cap) {
    const int P = pt->P;
    const std::vector<int32_t> l_ptr = download(pt->l_ptr, (size_t)pt->n + 1);
    const std::vector<int32_t> rr_ptr = download(pt->rr_ptr, (size_t)pt->n_rr + 1);
    const TileGeom g{32, cap, 2, 16, 1};
    std::vector<Tile> lt, rt;
    pt->lwtile_off.assign(P + 1, 0);
    pt->rwtile_off.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        pt->lwtile_off[p] = (int64_t)lt.size();
        tile_range(l_ptr, pt->bounds[p], pt->bounds[p + 1], (int32_t)pt->bounds[p], g, lt);
        pt->rwtile_off[p] = (int64_t)rt.size();
        tile_range(rr_ptr, pt->rr_off[p], pt->rr_off[p + 1], 0, g, rt);
    }
    pt->lwtile_off[P] = (int64_t)lt.size();
    pt->rwtile_off[P] = (int64_t)rt.size();
    free_one(pt, pt->lwtiles);
    free_one(pt, pt->rwtiles);
    pt->lwtiles = upload(pt, lt);
    pt->rwtiles = upload(pt, rt);
    pt->wtile_cap = cap;
}

// Sliced layout of one CSR (row pointer `ptr` over rows [0, rows)), rank p
// owning rows [rb[p], rb[p+1]) with x offset xo[p].  Per rank: rows longer
// than kSellLong go to the long list; the rest stay in natural order when
// padding every 32-position slice to its longest row adds at most 1/8 (+1024)
// entries, else they are sorted by length (descending, stable) behind the
// long rows.  Returns the padded entry count.
static int64_t build_sell_part(spmv_part* pt, spmv_part::SellPart& sp, const std::vector<int32_t>& ptr,
                               const std::vector<int64_t>& rb, const std::vector<int32_t>& xo,
                               const int32_t* d_ptr, const int32_t* d_col, const double* d_val) {
    const int P = pt->P;
    const int64_t rows = rb[P];
    std::vector<SellSlice> slices;
    std::vector<SellLong> longs;
    int64_t n_slots = 0, n_cut = 0;   // partial-sum slots and cut rows
    std::vector<uint8_t> len((size_t)rows, 0);
    std::vector<int32_t> perm;   // position -> row
    perm.reserve((size_t)rows);
    bool any_sorted = false;
    int64_t off = 0;
    sp.slice_off.assign(P + 1, 0);
    sp.long_off.assign(P + 1, 0);
    sp.sorted.assign(P, 0);
    std::vector<int32_t> order;
    for (int p = 0; p < P; ++p) {
        const int64_t r0 = rb[p], r1 = rb[p + 1];
        auto L = [&](int64_t r) { return ptr[(size_t)r + 1] - ptr[(size_t)r]; };
        // natural order: long rows are holes in their slices
        int64_t short_nnz = 0, nat = 0;
        for (int64_t r = r0; r < r1; r += 32) {
            int32_t mx = 0;
            for (int64_t i = r; i < std::min(r1, r + 32); ++i)
                if (L(i) <= kSellLong) mx = std::max(mx, L(i));
            nat += 32 * (int64_t)mx;
        }
        for (int64_t i = r0; i < r1; ++i)
            if (L(i) <= kSellLong) short_nnz += L(i);
        const bool sorted = nat > short_nnz + short_nnz / 8 + 1024;
        sp.sorted[p] = sorted;
        order.resize((size_t)(r1 - r0));
        for (int64_t i = r0; i < r1; ++i) order[(size_t)(i - r0)] = (int32_t)i;
        if (sorted) {
            any_sorted = true;
            std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return L(a) > L(b); });
        }
        perm.insert(perm.end(), order.begin(), order.end());   // identity for natural ranks
        sp.long_off[p] = (int64_t)longs.size();
        int64_t n_long_rows = 0;
        for (int64_t q = 0; q < r1 - r0; ++q) {
            const int32_t r = order[(size_t)q];
            if (L(r) > kSellLong) {
                ++n_long_rows;
                // pieces of at most kSellChunk entries, so that one very long
                // row does not keep one warp busy for the whole launch
                const int32_t kb = ptr[(size_t)r], ke = ptr[(size_t)r + 1];
                const int32_t np = (ke - kb + kSellChunk - 1) / kSellChunk;
                if (np == 1) {
                    longs.push_back(SellLong{r, xo[p], kb, ke, -1, -1, 1, -1});
                } else {
                    for (int32_t c = 0; c < np; ++c)
                        longs.push_back(SellLong{r, xo[p], kb + c * kSellChunk, std::min(ke, kb + (c + 1) * kSellChunk),
                                                 (int32_t)n_slots + c, (int32_t)n_slots, np, (int32_t)n_cut});
                    n_slots += np;
                    ++n_cut;
                }
            }
            len[(size_t)(r0 + q)] = L(r) > kSellLong ? kSellLenLong : (uint8_t)L(r);
        }
        // slices: sorted ranks skip their leading long rows
        const int64_t first = sorted ? r0 + n_long_rows : r0;
        sp.slice_off[p] = (int64_t)slices.size();
        for (int64_t q = first; q < r1; q += 32) {
            const int64_t e = std::min(r1, q + 32);
            int32_t mx = 0;
            for (int64_t i = q; i < e; ++i)
                if (len[(size_t)i] != kSellLenLong) mx = std::max<int32_t>(mx, len[(size_t)i]);
            if (off + 32 * (int64_t)mx > INT32_MAX - 64) fail(SPMV_EBOUNDS, "sliced layout exceeds 2^31 entries");
            slices.push_back(SellSlice{(int32_t)q, (int32_t)(e - q), mx, xo[p], (int32_t)off, 0, 0, 0});
            off += 32 * (int64_t)mx;
        }
    }
    sp.slice_off[P] = (int64_t)slices.size();
    sp.long_off[P] = (int64_t)longs.size();
    sp.h_slice_len.resize(slices.size());
    for (size_t i = 0; i < slices.size(); ++i) sp.h_slice_len[i] = slices[i].len;
    sp.h_long_len.resize(longs.size());
    for (size_t i = 0; i < longs.size(); ++i) sp.h_long_len[i] = longs[i].k1 - longs[i].k0;
    sp.slices = upload(pt, slices);
    sp.longs = upload(pt, longs);
    sp.long_part = static_cast<double*>(dev_alloc(pt, (size_t)n_slots * sizeof(double)));
    sp.long_cnt = static_cast<int*>(dev_alloc(pt, (size_t)n_cut * sizeof(int)));   // zeroed
    sp.len = upload(pt, len);
    sp.perm = any_sorted ? upload(pt, perm) : nullptr;
    sp.val = static_cast<double*>(dev_alloc(pt, (size_t)off * 8));
    sp.col = static_cast<int32_t*>(dev_alloc(pt, (size_t)off * 4));
    check_cuda(launch_sell_fill(d_ptr, d_col, d_val, sp.slices, (int)slices.size(), sp.len, sp.perm, sp.val, sp.col,
                                pt->num_sms, 0),
               "sliced layout");
    return off;
}

// Sliced-ELL copies of A_L and A_R (see build_sell_part), filled on the
// device from the plan's CSR arrays.
void build_sell(spmv_part* pt) {
    const int P = pt->P;
    const std::vector<int32_t> l_ptr = download(pt->l_ptr, (size_t)pt->n + 1);
    const std::vector<int32_t> rr_ptr = download(pt->rr_ptr, (size_t)pt->n_rr + 1);
    std::vector<int32_t> lxo(P), rxo(P, 0);
    for (int p = 0; p < P; ++p) lxo[p] = (int32_t)pt->bounds[p];
    pt->sell[0].entries = build_sell_part(pt, pt->sell[0], l_ptr, pt->bounds, lxo, pt->l_ptr, pt->l_col, pt->l_val);
    pt->sell[1].entries = build_sell_part(pt, pt->sell[1], rr_ptr, pt->rr_off, rxo, pt->rr_ptr, pt->r_col, pt->r_val);
    // the remote product's y row of each position in one table, so that a
    // sorted slice's store reads one coalesced index instead of its row and
    // then the scattered row map
    spmv_part::SellPart& sr = pt->sell[1];
    if (sr.perm) {
        const std::vector<int32_t> rr_row = download(pt->rr_row, (size_t)pt->n_rr);
        const std::vector<int32_t> perm = download(sr.perm, (size_t)pt->n_rr);
        std::vector<int32_t> ypos((size_t)pt->n_rr);
        for (size_t q = 0; q < ypos.size(); ++q) ypos[q] = rr_row[(size_t)perm[q]];
        sr.ypos = upload(pt, ypos);
    }
    check_cuda(cudaDeviceSynchronize(), "sliced layout");
    pt->sell_entries = pt->sell[0].entries + pt->sell[1].entries;
    pt->sell_built = true;
}

// Cost-balanced CTA ranges of the sliced launches of part_idx (0 LOCAL, 1
// REMOTE) at `param`, for every launch site: a site's units (its long-row
// pieces, then its slices, the order the kernel numbers them) are cut into
// sell_grid(...) contiguous ranges of about equal estimated cost, so each CTA
// (and so each SM, which holds several) gets the same work and keeps the
// neighbouring slices of the round-robin split together.  A unit's cost is
// its entries per lane (a slice's longest row; a piece's entries over 32,
// rounded up) plus 3 for its descriptor, row and store.
// Estimated time of one work unit of a sliced launch: a fixed part (the
// unit's descriptor, lengths and row-map loads and its stores) plus one per
// entry of a lane (slots of a slice lane; a long-row piece's entries over
// 32 lanes).  Measured against costs by dependent rounds (2 + 2 rounds +
// entries / 4, and 1 + rounds) on the power-law matrix's per-rank launches,
// this one balanced best.
double sell_unit_cost(bool long_piece, int64_t len) {
    const int64_t per_lane = long_piece ? (len + 31) / 32 : len;
    return 3.0 + (double)per_lane;
}

void build_sell_split(spmv_part* pt, int part_idx, int param) {
    spmv_part::SellPart& sp = pt->sell[part_idx];
    const int P = pt->P;
    for (int site = 0; site <= P; ++site) {
        const int64_t lb = site < P ? sp.long_off[site] : 0, le = site < P ? sp.long_off[site + 1] : sp.long_off[P];
        const int64_t sb = site < P ? sp.slice_off[site] : 0, se = site < P ? sp.slice_off[site + 1] : sp.slice_off[P];
        const int units = (int)((le - lb) + (se - sb));
        const int grid = sell_grid(param, units, pt->num_sms);
        if (grid <= 0) continue;
        const int64_t key = ((int64_t)site << 32) | grid;
        if (sp.cta_split.count(key)) continue;
        std::vector<double> prefix((size_t)units + 1, 0.0);
        for (int u = 0; u < units; ++u) {
            const bool lng = u < le - lb;
            const int64_t len = lng ? sp.h_long_len[(size_t)(lb + u)] : sp.h_slice_len[(size_t)(sb + u - (le - lb))];
            prefix[(size_t)u + 1] = prefix[(size_t)u] + sell_unit_cost(lng, len);
        }
        std::vector<int32_t> off((size_t)grid + 1);
        const double total = prefix[(size_t)units];
        for (int b = 0; b <= grid; ++b) {
            const double target = total * b / grid;
            off[(size_t)b] = (int32_t)(std::lower_bound(prefix.begin(), prefix.end(), target) - prefix.begin());
        }
        off[0] = 0;
        off[(size_t)grid] = units;
        for (int b = 1; b <= grid; ++b) off[(size_t)b] = std::max(off[(size_t)b], off[(size_t)b - 1]);
        sp.cta_split[key] = upload(pt, off);
    }
}

const int32_t* sell_split(const spmv_part* pt, int part_idx, int site, int grid) {
    const spmv_part::SellPart& sp = pt->sell[part_idx];
    auto it = sp.cta_split.find(((int64_t)site << 32) | grid);
    return it == sp.cta_split.end() ? nullptr : it->second;
}

// Release of the CSR copy once both products use the sliced layout: each
// layout's long rows (which the sliced kernel reads from the CSR) move to
// compact arrays of their own, piece after piece, and the pieces are
// re-pointed at them; then the CSR columns and values of A_L and A_R are
// freed, and the 32-bit slot columns of A_L too when its product uses the
// 16-bit deltas.  Row pointers stay.  restore_csr undoes all of it on the
// device: slots back into their rows, long rows back, pieces re-pointed.
void release_csr(spmv_part* pt) {
    if (pt->csr_released) return;
    const bool sliced0 = pt->variant[0] == SPMV_VARIANT_SELL || pt->variant[0] == SPMV_VARIANT_SELL16;
    const bool sliced1 = pt->variant[1] == SPMV_VARIANT_SELL;
    if (!pt->sell_built || !sliced0 || !sliced1)
        fail(SPMV_EINVAL, "both products must use the sliced layout before the CSR copy is released");
    check_cuda(cudaDeviceSynchronize(), "synchronize");
    const int P = pt->P;
    for (int i = 0; i < 2; ++i) {
        spmv_part::SellPart& sp = pt->sell[i];
        const int nl = (int)sp.long_off[P];
        std::vector<SellLong> L = download(sp.longs, (size_t)nl);
        std::vector<int32_t> tab((size_t)3 * nl);
        sp.h_long_csr_k0.assign((size_t)nl, 0);
        int64_t c = 0;
        for (int j = 0; j < nl; ++j) {
            const int32_t len = L[(size_t)j].k1 - L[(size_t)j].k0;
            tab[(size_t)3 * j] = L[(size_t)j].k0;
            tab[(size_t)3 * j + 1] = (int32_t)c;
            tab[(size_t)3 * j + 2] = len;
            sp.h_long_csr_k0[(size_t)j] = L[(size_t)j].k0;
            L[(size_t)j].k0 = (int32_t)c;
            L[(size_t)j].k1 = (int32_t)(c + len);
            c += len;
        }
        if (nl > 0) {
            sp.long_val = static_cast<double*>(dev_alloc(pt, (size_t)c * 8));
            sp.long_col = static_cast<int32_t*>(dev_alloc(pt, (size_t)c * 4));
            int32_t* d_tab = upload(pt, tab);
            check_cuda(launch_segment_copy(d_tab, nl, i ? pt->r_val : pt->l_val, i ? pt->r_col : pt->l_col,
                                           sp.long_val, sp.long_col, pt->num_sms, 0),
                       "long rows out of the CSR");
            check_cuda(cudaMemcpy(sp.longs, L.data(), (size_t)nl * sizeof(SellLong), cudaMemcpyHostToDevice),
                       "long-row pieces");
            check_cuda(cudaDeviceSynchronize(), "long rows out of the CSR");
            free_one(pt, d_tab);
        }
    }
    free_one(pt, pt->l_col);
    free_one(pt, pt->l_val);
    free_one(pt, pt->r_col);
    free_one(pt, pt->r_val);
    pt->l_col = pt->r_col = nullptr;
    pt->l_val = pt->r_val = nullptr;
    if (pt->variant[0] == SPMV_VARIANT_SELL16 && pt->sell[0].col16) {
        free_one(pt, pt->sell[0].col);
        pt->sell[0].col = nullptr;
    }
    pt->csr_released = true;
}

void restore_csr(spmv_part* pt) {
    if (!pt->csr_released) return;
    check_cuda(cudaDeviceSynchronize(), "synchronize");
    const int P = pt->P;
    pt->l_col = static_cast<int32_t*>(dev_alloc(pt, (size_t)pt->nnz_l * 4));
    pt->l_val = static_cast<double*>(dev_alloc(pt, (size_t)pt->nnz_l * 8));
    pt->r_col = static_cast<int32_t*>(dev_alloc(pt, (size_t)pt->nnz_r * 4));
    pt->r_val = static_cast<double*>(dev_alloc(pt, (size_t)pt->nnz_r * 8));
    for (int i = 0; i < 2; ++i) {
        spmv_part::SellPart& sp = pt->sell[i];
        int32_t* col = i ? pt->r_col : pt->l_col;
        double* val = i ? pt->r_val : pt->l_val;
        check_cuda(launch_sell_unfill(i ? pt->rr_ptr : pt->l_ptr, sp.slices, (int)sp.slice_off[P], sp.len, sp.perm,
                                      sp.val, sp.col, sp.col16, col, val, pt->num_sms, 0),
                   "slots back into the CSR");
        const int nl = (int)sp.long_off[P];
        if (nl > 0) {
            std::vector<SellLong> L = download(sp.longs, (size_t)nl);
            std::vector<int32_t> tab((size_t)3 * nl);
            for (int j = 0; j < nl; ++j) {
                const int32_t len = L[(size_t)j].k1 - L[(size_t)j].k0;
                tab[(size_t)3 * j] = L[(size_t)j].k0;
                tab[(size_t)3 * j + 1] = sp.h_long_csr_k0[(size_t)j];
                tab[(size_t)3 * j + 2] = len;
                L[(size_t)j].k0 = sp.h_long_csr_k0[(size_t)j];
                L[(size_t)j].k1 = L[(size_t)j].k0 + len;
            }
            int32_t* d_tab = upload(pt, tab);
            check_cuda(launch_segment_copy(d_tab, nl, sp.long_val, sp.long_col, val, col, pt->num_sms, 0),
                       "long rows back into the CSR");
            check_cuda(cudaMemcpy(sp.longs, L.data(), (size_t)nl * sizeof(SellLong), cudaMemcpyHostToDevice),
                       "long-row pieces");
            check_cuda(cudaDeviceSynchronize(), "long rows back into the CSR");
            free_one(pt, d_tab);
            free_one(pt, sp.long_val);
            free_one(pt, sp.long_col);
            sp.long_val = nullptr;
            sp.long_col = nullptr;
        }
        sp.h_long_csr_k0.clear();
    }
    spmv_part::SellPart& s0 = pt->sell[0];
    if (!s0.col) {
        s0.col = static_cast<int32_t*>(dev_alloc(pt, (size_t)s0.entries * 4));
        check_cuda(launch_sell_col32(s0.slices, (int)s0.slice_off[P], s0.len, s0.perm, s0.col16, s0.col, pt->num_sms,
                                     0),
                   "32-bit slot columns");
    }
    check_cuda(cudaDeviceSynchronize(), "CSR restored");
    pt->csr_released = false;
}

// 16-bit column deltas of the LOCAL sliced layout (built on first use);
// false when some |column - row| needs more than 16 bits.
bool build_sell_delta16(spmv_part* pt) {
    spmv_part::SellPart& sp = pt->sell[0];
    if (sp.delta_state != 0) return sp.delta_state > 0;
    int16_t* c16 = static_cast<int16_t*>(dev_alloc(pt, (size_t)sp.entries * 2));
    int* bad = static_cast<int*>(dev_alloc(pt, sizeof(int)));
    const int n_slices = (int)sp.slice_off[pt->P];
    check_cuda(launch_sell_delta(sp.slices, n_slices, sp.len, sp.perm, sp.col, c16, bad, pt->num_sms, 0),
               "column deltas");
    int h = 0;
    check_cuda(cudaMemcpy(&h, bad, sizeof(int), cudaMemcpyDeviceToHost), "column deltas");
    free_one(pt, bad);
    if (h) {
        free_one(pt, c16);
        sp.delta_state = -1;
        return false;
    }
    sp.col16 = c16;
    sp.delta_state = 1;
    return true;
}

}  // namespace spmvk
