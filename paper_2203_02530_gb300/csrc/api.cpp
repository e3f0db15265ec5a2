// C ABI of the partitioned SpMV library (include/spmv.h): plan life cycle,
// the four operations of Fig. 3c, and the schedule runner of Sec. III-B with
// Table III synchronisation, eager or captured as a CUDA graph.
#include "part.h"
#include "pdl.cuh"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

using spmvk::fail;
using spmvk::check_cuda;

namespace {

thread_local std::string g_err;

// Test hook of the plan-free merge entry points (spmv_selftest_merge_abort):
// tile + 1 from which their merge kernel takes the give-up path, 0 = never.
std::atomic<int> g_merge_abort_tile{0};

int fail_status(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

}  // namespace

void spmvk::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

#define API_TRY try {
#define API_CATCH                                                                         \
    }                                                                                     \
    catch (const spmvk::Fail& f) {                                                        \
        return fail_status(f.code, f.msg);                                                \
    }                                                                                     \
    catch (const std::bad_alloc&) {                                                       \
        return fail_status(SPMV_ENOMEM, "host allocation failed");                        \
    }                                                                                     \
    catch (...) {                                                                         \
        return fail_status(SPMV_EINVAL, "unexpected exception");                          \
    }

void need(bool ok, int code, const char* msg) {
    if (!ok) fail(code, "%s", msg);
}

void check_part(const spmv_part* pt) { need(pt != nullptr, SPMV_EINVAL, "part is NULL"); }

void check_rank(const spmv_part* pt, int part_idx) {
    if (part_idx < -1 || part_idx >= pt->P) fail(SPMV_EINVAL, "part index %d not in [-1, %d)", part_idx, pt->P);
}

// The operations' DAG (Fig. 3c): pack -> copy -> remote, local -> remote;
// per rank, pack of q -> copy of p whenever q sends to p.
void build_dag(spmv_part* pt) {
    const int P = pt->P;
    pt->edges.clear();
    if (pt->gran == SPMV_COARSE) {
        pt->n_ops = 4;
        pt->edges = {{SPMV_OP_PACK, SPMV_OP_COPY}, {SPMV_OP_COPY, SPMV_OP_REMOTE},
                     {SPMV_OP_LOCAL, SPMV_OP_REMOTE}};
    } else if (pt->gran == SPMV_PER_SEGMENT) {
        // ops 2p (LOCAL of rank p), 2p+1 (REMOTE of rank p), then for every
        // nonempty segment k: 2P+2k (its PACK), 2P+2k+1 (its COPY)
        pt->segs.clear();
        for (int p = 0; p < P; ++p)
            for (int q = 0; q < P; ++q) {
                const int64_t a = pt->seg_off[(size_t)p * P + q], b = pt->seg_off[(size_t)p * P + q + 1];
                if (q != p && b > a) pt->segs.push_back(spmv_part::Seg{p, q, a, b});
            }
        pt->n_ops = 2 * P + 2 * (int)pt->segs.size();
        for (int p = 0; p < P; ++p) pt->edges.push_back({2 * p, 2 * p + 1});
        for (size_t k = 0; k < pt->segs.size(); ++k) {
            const int pack = 2 * P + 2 * (int)k;
            pt->edges.push_back({pack, pack + 1});
            pt->edges.push_back({pack + 1, 2 * pt->segs[k].p + 1});
        }
    } else {
        pt->n_ops = 4 * P;
        for (int p = 0; p < P; ++p) {
            for (int q = 0; q < P; ++q) {
                if (q == p) continue;
                if (pt->seg_off[(size_t)p * P + q + 1] > pt->seg_off[(size_t)p * P + q])
                    pt->edges.push_back({4 * q + SPMV_OP_PACK, 4 * p + SPMV_OP_COPY});
            }
            pt->edges.push_back({4 * p + SPMV_OP_COPY, 4 * p + SPMV_OP_REMOTE});
            pt->edges.push_back({4 * p + SPMV_OP_LOCAL, 4 * p + SPMV_OP_REMOTE});
        }
    }
    pt->preds.assign(pt->n_ops, {});
    for (auto& e : pt->edges) pt->preds[e.second].push_back(e.first);
}

spmvk::CsrArgs local_args(spmv_part* pt, const double* x, double* y) {
    spmvk::CsrArgs a{};
    a.ptr = pt->l_ptr;
    a.col = pt->l_col;
    a.val = pt->l_val;
    a.rowmap = nullptr;
    a.x = x;
    a.y = y;
    a.accumulate = 0;
    a.n_rows = (int)pt->n;
    a.nnz_total = (int)pt->nnz_l;
    a.guarded = 0;
    a.err = pt->err;
    a.pdl = pt->cur_pdl;
    return a;
}

spmvk::CsrArgs remote_args(spmv_part* pt, double* y) {
    spmvk::CsrArgs a{};
    a.ptr = pt->rr_ptr;
    a.col = pt->r_col;
    a.val = pt->r_val;
    a.rowmap = pt->rr_row;
    a.x = pt->recvbuf;
    a.y = y;
    a.accumulate = 1;
    a.n_rows = (int)pt->n_rr;
    a.nnz_total = (int)pt->nnz_r;
    a.guarded = 0;
    a.err = pt->err;
    a.pdl = pt->cur_pdl;
    return a;
}

// Each op returns the number of kernels it launched.
int op_pack(spmv_part* pt, int q, const double* x, cudaStream_t s) {
    if (q < 0) {
        if (pt->dry_run) return pt->n_send > 0;
        check_cuda(spmvk::launch_gather(x, pt->send_idx, nullptr, pt->sendbuf, pt->n_send, pt->num_sms, s,
                                        pt->cur_pdl),
                   "pack");
        return pt->n_send > 0;
    }
    const int64_t c = pt->pack_off[q + 1] - pt->pack_off[q];
    if (pt->dry_run) return c > 0;
    check_cuda(spmvk::launch_gather(x, pt->send_idx, pt->pack_pos + pt->pack_off[q], pt->sendbuf, c,
                                    pt->num_sms, s, pt->cur_pdl),
               "pack");
    return c > 0;
}

int op_copy(spmv_part* pt, int p, cudaStream_t s) {
    const int64_t a = p < 0 ? 0 : pt->halo_off[p];
    const int64_t b = p < 0 ? pt->n_send : pt->halo_off[p + 1];
    if (pt->dry_run) return b > a;
    check_cuda(spmvk::launch_copy(pt->sendbuf + a, pt->recvbuf + a, b - a, pt->num_sms, s, pt->cur_pdl), "halo copy");
    return b > a;
}

int launch_product(spmv_part* pt, const spmvk::CsrArgs& a, bool remote, int p, cudaStream_t s) {
    const std::vector<int64_t>& off = remote ? pt->rtile_off : pt->ltile_off;
    const int tb = (int)(p < 0 ? 0 : off[p]);
    const int te = (int)(p < 0 ? off[pt->P] : off[p + 1]);
    const int var = pt->variant[remote ? 1 : 0];
    const int param = pt->vparam[remote ? 1 : 0];
    if (var == SPMV_VARIANT_MERGE) {
        const std::vector<int64_t>& mo = remote ? pt->rmtile_off : pt->lmtile_off;
        const int mb = (int)(p < 0 ? 0 : mo[p]);
        const int me = (int)(p < 0 ? mo[pt->P] : mo[p + 1]);
        if (pt->dry_run) return me > mb ? 2 : 0;
        check_cuda(spmvk::launch_merge(a, remote ? pt->rmtiles : pt->lmtiles, mb, me,
                                       remote ? pt->rcarry : pt->lcarry, pt->num_sms, s),
                   "merge product");
        return me > mb ? 2 : 0;
    }
    if (var == SPMV_VARIANT_WARP) {
        const std::vector<int64_t>& wo = remote ? pt->rwtile_off : pt->lwtile_off;
        const int wb = (int)(p < 0 ? 0 : wo[p]);
        const int we = (int)(p < 0 ? wo[pt->P] : wo[p + 1]);
        if (pt->dry_run) return we > wb;
        check_cuda(spmvk::launch_warp(a, remote ? pt->rwtiles : pt->lwtiles, wb, we, param, pt->num_sms, s),
                   "warp product");
        return we > wb;
    }
    if (var == SPMV_VARIANT_SELL || var == SPMV_VARIANT_SELL16) {
        const spmv_part::SellPart& sp = pt->sell[remote ? 1 : 0];
        spmvk::SellArgs sa{sp.slices, sp.longs, sp.val,  sp.col,         sp.col16,     sp.len, sp.perm,
                           0,         0,        0,       0,       sp.long_part, sp.long_cnt, nullptr};
        sa.ypos = sp.ypos;
        sa.slice_begin = (int)(p < 0 ? 0 : sp.slice_off[p]);
        sa.slice_end = (int)(p < 0 ? sp.slice_off[pt->P] : sp.slice_off[p + 1]);
        sa.long_begin = (int)(p < 0 ? 0 : sp.long_off[p]);
        sa.long_end = (int)(p < 0 ? sp.long_off[pt->P] : sp.long_off[p + 1]);
        if (pt->dry_run) return (sa.slice_end > sa.slice_begin || sa.long_end > sa.long_begin) ? 1 : 0;
        if (spmvk::sell_param_balanced(param)) {
            const int units = (sa.slice_end - sa.slice_begin) + (sa.long_end - sa.long_begin);
            const int grid = spmvk::sell_grid(param, units, pt->num_sms);
            if (grid > 0) {
                sa.cta_off = spmvk::sell_split(pt, remote ? 1 : 0, p < 0 ? pt->P : p, grid);
                if (!sa.cta_off) fail(SPMV_EINVAL, "balanced sliced ranges not prepared");
            }
        }
        spmvk::CsrArgs al = a;   // long rows: from the CSR, or its compact copy once the CSR is released
        if (sp.long_col) {
            al.col = sp.long_col;
            al.val = sp.long_val;
        }
        check_cuda(spmvk::launch_sell(al, sa, param, var == SPMV_VARIANT_SELL16, pt->num_sms, s), "sliced product");
        return (sa.slice_end > sa.slice_begin || sa.long_end > sa.long_begin) ? 1 : 0;
    }
    const spmvk::Tile* tiles = remote ? pt->rtiles : pt->ltiles;
    if (var == SPMV_VARIANT_VECTOR || var == SPMV_VARIANT_PAIRS) {
        const std::vector<int64_t>& bo = remote ? pt->rblock_off : pt->lblock_off;
        const int bb = (int)(p < 0 ? 0 : bo[p]);
        const int be = (int)(p < 0 ? bo[pt->P] : bo[p + 1]);
        const spmvk::Tile* blocks = remote ? pt->rblocks : pt->lblocks;
        if (pt->dry_run) return be > bb;
        if (var == SPMV_VARIANT_VECTOR)
            check_cuda(spmvk::launch_vector(a, blocks, bb, be, param, pt->num_sms, s), "vector product");
        else
            check_cuda(spmvk::launch_pairs(a, blocks, bb, be, param, pt->num_sms, s), "pair product");
        return be > bb;
    } else {
        if (pt->dry_run) return te > tb;
        check_cuda(spmvk::launch_tile(a, tiles, tb, te, pt->geom, pt->num_sms, s), "tile product");
    }
    return te > tb;
}

int op_local(spmv_part* pt, int p, const double* x, double* y, cudaStream_t s) {
    return launch_product(pt, local_args(pt, x, y), false, p, s);
}

int op_remote(spmv_part* pt, int p, double* y, cudaStream_t s) {
    return launch_product(pt, remote_args(pt, y), true, p, s);
}

// PACK of one halo segment: its send slots [a, b) <- x
int op_pack_segment(spmv_part* pt, const spmv_part::Seg& g, const double* x, cudaStream_t s) {
    if (pt->dry_run) return g.b > g.a;
    check_cuda(spmvk::launch_gather(x, pt->send_idx + g.a, nullptr, pt->sendbuf + g.a, g.b - g.a, pt->num_sms, s,
                                    pt->cur_pdl),
               "pack segment");
    return g.b > g.a;
}

// COPY of one halo segment: recvbuf[a, b) <- sendbuf[a, b)
int op_copy_segment(spmv_part* pt, const spmv_part::Seg& g, cudaStream_t s) {
    if (pt->dry_run) return g.b > g.a;
    check_cuda(spmvk::launch_copy(pt->sendbuf + g.a, pt->recvbuf + g.a, g.b - g.a, pt->num_sms, s, pt->cur_pdl),
               "copy segment");
    return g.b > g.a;
}

int run_op(spmv_part* pt, int op, const double* x, double* y, cudaStream_t s) {
    if (pt->gran == SPMV_PER_SEGMENT) {
        const int P = pt->P;
        if (op < 2 * P) return op % 2 == 0 ? op_local(pt, op / 2, x, y, s) : op_remote(pt, op / 2, y, s);
        const spmv_part::Seg& g = pt->segs[(size_t)(op - 2 * P) / 2];
        return (op - 2 * P) % 2 == 0 ? op_pack_segment(pt, g, x, s) : op_copy_segment(pt, g, s);
    }
    const int kind = op % 4;
    const int p = pt->gran == SPMV_COARSE ? -1 : op / 4;
    switch (kind) {
        case SPMV_OP_PACK: return op_pack(pt, p, x, s);
        case SPMV_OP_LOCAL: return op_local(pt, p, x, y, s);
        case SPMV_OP_COPY: return op_copy(pt, p, s);
        default: return op_remote(pt, p, y, s);
    }
}

void validate_schedule(const spmv_part* pt, const int32_t* order, const int32_t* stream_of, int n_ops,
                       int n_streams) {
    if (!order || !stream_of) fail(SPMV_EINVAL, "op_order or stream_of_op is NULL");
    if (n_ops != pt->n_ops) fail(SPMV_ESCHED, "%d ops given, the DAG has %d", n_ops, pt->n_ops);
    if (n_streams < 1) fail(SPMV_EINVAL, "n_streams = %d", n_streams);
    std::vector<int> pos(n_ops, -1);
    for (int i = 0; i < n_ops; ++i) {
        const int v = order[i];
        if (v < 0 || v >= n_ops) fail(SPMV_ESCHED, "op id %d out of range", v);
        if (pos[v] >= 0) fail(SPMV_ESCHED, "op %d appears twice", v);
        pos[v] = i;
    }
    for (int v = 0; v < n_ops; ++v)
        if (stream_of[v] < 0 || stream_of[v] >= n_streams)
            fail(SPMV_ESCHED, "op %d bound to stream %d of %d", v, stream_of[v], n_streams);
    for (auto& e : pt->edges)
        if (pos[e.first] > pos[e.second])
            fail(SPMV_ESCHED, "order is not topological: op %d must precede op %d", e.first, e.second);
}

void ensure_events(spmv_part* pt, int n_streams) {
    if (pt->op_ev.empty()) {
        pt->op_ev.assign(pt->n_ops, nullptr);
        for (auto& e : pt->op_ev) check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        check_cuda(cudaEventCreateWithFlags(&pt->fork_ev, cudaEventDisableTiming), "event");
    }
    while ((int)pt->join_ev.size() < n_streams) {
        cudaEvent_t e;
        check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        pt->join_ev.push_back(e);
    }
}

// Issue one implementation (order + stream map) with Table III events.
// Relaxed mode (SPMV_RUN_RELAXED, captured graphs only): an op with no DAG
// predecessor (a pack or a local product) skips the programmatic wait for
// the kernel before it on its stream (kPdlNoWait), and that kernel releases
// it as its CTAs start (kPdlEarly), so the two overlap.  Every other op waits
// as in the default mode (griddepcontrol.wait: all of its kernel's
// prerequisite nodes complete), and every DAG edge, also between two ops of
// one stream, is an event recorded after its source and waited for before
// its target, so an op's predecessors are always among its prerequisites
// even when a kernel between them on the stream did not wait.
// Deferred mode (SPMV_RUN_DEFER, stream semantics otherwise): a remote
// product in the sliced layout whose kernel follows, on its stream, a kernel
// that writes none of its inputs but y (any op that is not its DAG
// predecessor, or its local product) reads A_R and the halo and sums its
// rows before waiting for that kernel, and waits only before its first
// access to y (kPdlDefer); that kernel releases it as its CTAs start, after
// its own wait (kPdlEarly).  Every kernel before that one on the stream is
// then complete, and the remote product's other predecessors are on other
// streams, behind events whose graph edges are made full dependencies after
// capture (fix_deferred_edges).  With the relaxed mode as well, the kernel
// before it may not have waited (an op without DAG predecessors), but every
// DAG edge is then an event, so the remote product's predecessors other
// than that kernel are again behind full edges.
int op_kind(const spmv_part* pt, int op) {
    if (pt->gran == SPMV_COARSE) return op;
    if (pt->gran == SPMV_PER_PARTITION) return op % 4;
    if (op < 2 * pt->P) return op % 2 == 0 ? SPMV_OP_LOCAL : SPMV_OP_REMOTE;
    return (op - 2 * pt->P) % 2 == 0 ? SPMV_OP_PACK : SPMV_OP_COPY;
}

void defer_flags(spmv_part* pt, const int32_t* order, const int32_t* stream_of, int n_ops, int n_streams,
                 const double* x, double* y, cudaStream_t s, std::vector<int>& pdl_flags) {
    const int rv = pt->variant[1];
    if (rv != SPMV_VARIANT_SELL && rv != SPMV_VARIANT_SELL16) return;
    // kernels each op launches (an op with nothing to do launches none, and
    // the kernel before it on the stream is then the one that releases)
    std::vector<int> kernels(n_ops, 0);
    pt->dry_run = true;
    try {
        for (int v = 0; v < n_ops; ++v) kernels[v] = run_op(pt, v, x, y, s);
    } catch (...) {
        pt->dry_run = false;
        throw;
    }
    pt->dry_run = false;
    std::vector<int> last(n_streams, -1);   // last op of each stream that launched a kernel
    for (int i = 0; i < n_ops; ++i) {
        const int v = order[i];
        const int u = last[stream_of[v]];
        if (kernels[v] > 0 && u >= 0 && op_kind(pt, v) == SPMV_OP_REMOTE) {
            bool feeds = false;   // u writes an input of v other than y
            for (int w : pt->preds[v])
                if (w == u && op_kind(pt, u) != SPMV_OP_LOCAL) feeds = true;
            if (!feeds) {
                pdl_flags[v] |= spmvk::kPdlDefer;
                pdl_flags[u] |= spmvk::kPdlEarly;
            }
        }
        if (kernels[v] > 0) last[stream_of[v]] = v;
    }
}

void issue(spmv_part* pt, const int32_t* order, const int32_t* stream_of, int n_ops, cudaStream_t* streams,
           int n_streams, const double* x, double* y, bool relaxed, bool defer) {
    std::vector<int> pdl_flags(n_ops, 0);
    if (defer) defer_flags(pt, order, stream_of, n_ops, n_streams, x, y, streams[0], pdl_flags);
    if (relaxed) {
        std::vector<int> last(n_streams, -1);
        for (int i = 0; i < n_ops; ++i) {
            const int v = order[i];
            const bool free_op = pt->preds[v].empty();
            if (free_op) {
                pdl_flags[v] |= spmvk::kPdlNoWait;
                if (last[stream_of[v]] >= 0) pdl_flags[last[stream_of[v]]] |= spmvk::kPdlEarly;
            }
            last[stream_of[v]] = v;
        }
    }
    cudaStream_t origin = streams[0];
    std::vector<char> used(n_streams, 0);
    for (int v = 0; v < n_ops; ++v) used[stream_of[v]] = 1;
    // start vertex: fork every other used stream from the origin
    check_cuda(cudaEventRecord(pt->fork_ev, origin), "fork record");
    for (int s = 1; s < n_streams; ++s)
        if (used[s]) check_cuda(cudaStreamWaitEvent(streams[s], pt->fork_ev, 0), "fork wait");
    // which ops feed a successor bound to another stream (any successor in
    // relaxed mode)
    std::vector<char> cross(n_ops, 0);
    for (auto& e : pt->edges)
        if (relaxed || stream_of[e.first] != stream_of[e.second]) cross[e.first] = 1;
    int64_t records = 0, waits = 0, launches = 0;
    // while capturing a deferred program: the last kernel node of each stream
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (defer) check_cuda(cudaStreamIsCapturing(origin, &cap), "capture status");
    const bool track = defer && cap == cudaStreamCaptureStatusActive;
    std::vector<cudaGraphNode_t> last_node(n_streams, nullptr);
    pt->deferred_nodes.clear();
    for (int i = 0; i < n_ops; ++i) {
        const int v = order[i];
        cudaStream_t sv = streams[stream_of[v]];
        for (int u : pt->preds[v]) {
            if (relaxed || stream_of[u] != stream_of[v]) {   // Table III: BoundGPU_i -> BoundGPU_j
                check_cuda(cudaStreamWaitEvent(sv, pt->op_ev[u], 0), "stream wait");
                ++waits;
            }                                                // same stream: nothing
        }
        int k = 0;
        {
            pt->cur_pdl = pdl_flags[v];
            try {
                k = run_op(pt, v, x, y, sv);
            } catch (...) {
                pt->cur_pdl = 0;
                throw;
            }
            pt->cur_pdl = 0;
            launches += k;
        }
        if (track && k > 0) {
            // the stream's capture dependency is now the op's last kernel
            cudaStreamCaptureStatus st;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            check_cuda(cudaStreamGetCaptureInfo(sv, &st, nullptr, nullptr, &deps, nullptr, &nd), "capture info");
            if (nd != 1) fail(SPMV_EINVAL, "unexpected capture dependencies (%zu) after an op", nd);
            if (pdl_flags[v] & spmvk::kPdlDefer) pt->deferred_nodes.push_back({deps[0], last_node[stream_of[v]]});
            last_node[stream_of[v]] = deps[0];
        }
        if (cross[v]) {
            check_cuda(cudaEventRecord(pt->op_ev[v], sv), "event record");
            ++records;
        }
    }
    // end vertex: join every other used stream back into the origin
    for (int s = 1; s < n_streams; ++s) {
        if (!used[s]) continue;
        check_cuda(cudaEventRecord(pt->join_ev[s], streams[s]), "join record");
        check_cuda(cudaStreamWaitEvent(origin, pt->join_ev[s], 0), "join wait");
    }
    pt->last_records = records;
    pt->last_waits = waits;
    pt->last_launches = launches;
    pt->last_deferred = 0;
    for (int v = 0; v < n_ops; ++v) pt->last_deferred += (pdl_flags[v] & spmvk::kPdlDefer) != 0;
}

int64_t alg_bytes_local(const spmv_part* pt) {
    // 12 B per entry, 4 B per row pointer (+1), 8 B x read, 8 B y written
    return 12 * pt->nnz_l + 4 * (pt->n + 1) + 8 * pt->n + 8 * pt->n;
}

int64_t alg_bytes_total(const spmv_part* pt) {
    // local product, the remote product (entries, compressed row pointers
    // and row ids, y read-modify-write of its rows), the pack (indices read,
    // slots written; its x reads are counted in the local product's x),
    // the exchange (read + write) and the remote product's halo reads
    int64_t b = alg_bytes_local(pt);
    b += 12 * pt->nnz_r + 4 * (pt->n_rr + 1) + 4 * pt->n_rr + 16 * pt->n_rr;
    b += 4 * pt->n_send + 8 * pt->n_send;   // pack: index read, slot write
    b += 16 * pt->n_send;                   // exchange: read + write
    b += 8 * pt->n_send;                    // remote: halo read
    return b;
}

template <class T>
std::vector<T> d2h(const T* d, int64_t count) {
    std::vector<T> h((size_t)std::max<int64_t>(count, 0));
    if (count > 0) check_cuda(cudaMemcpy(h.data(), d, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost), "export");
    return h;
}

// Stream capture gives every incoming edge of a kernel launched with
// programmatic stream serialization the programmatic type, the edges of its
// cross-stream event waits included (a kernel that waits at its start waits
// for all of them alike).  A deferred remote product reads A_R and the halo
// before its wait, so only the edge from the kernel before it on its stream
// may stay programmatic: every other incoming edge of its node becomes a
// full dependency (completion and memory visibility), and the result is
// checked before the graph is instantiated.
bool edge_is_default(const cudaGraphEdgeData& e) { return e.type == 0 && e.from_port == 0 && e.to_port == 0; }

void fix_deferred_edges(const spmv_part* pt, cudaGraph_t g) {
    const cudaGraphEdgeData full{};
    for (const auto& dn : pt->deferred_nodes) {
        const cudaGraphNode_t v = dn.first, u = dn.second;
        for (int pass = 0; pass < 2; ++pass) {   // rewrite, then check
            size_t nd = 0;
            check_cuda(cudaGraphNodeGetDependencies(v, nullptr, nullptr, &nd), "node dependencies");
            std::vector<cudaGraphNode_t> from(nd);
            std::vector<cudaGraphEdgeData> ed(nd);
            if (nd) check_cuda(cudaGraphNodeGetDependencies(v, from.data(), ed.data(), &nd), "node dependencies");
            int from_u = 0;
            for (size_t i = 0; i < nd; ++i) {
                if (from[i] == u) {
                    ++from_u;
                } else if (!edge_is_default(ed[i])) {
                    if (pass == 1) fail(SPMV_EINVAL, "a deferred remote product kept a programmatic edge");
                    check_cuda(cudaGraphRemoveDependencies(g, &from[i], &v, &ed[i], 1), "remove edge");
                    check_cuda(cudaGraphAddDependencies(g, &from[i], &v, &full, 1), "add edge");
                }
            }
            if (from_u != 1) fail(SPMV_EINVAL, "a deferred remote product lost the edge from its stream predecessor");
        }
    }
}

}  // namespace

extern "C" {

int spmv_part_create(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* vals, int P,
                     int granularity, spmv_part** out) {
    if (!out) return fail_status(SPMV_EINVAL, "out is NULL");
    *out = nullptr;
    spmv_part* pt = nullptr;
    API_TRY
    if (granularity != SPMV_COARSE && granularity != SPMV_PER_PARTITION && granularity != SPMV_PER_SEGMENT)
        fail(SPMV_EINVAL, "granularity %d", granularity);
    spmvk::validate_csr(n, row_ptr, col_idx, vals, P);   // before any CUDA call
    pt = new spmv_part();
    pt->P = P;
    pt->gran = granularity;
    check_cuda(cudaGetDevice(&pt->device), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&pt->num_sms, cudaDevAttrMultiProcessorCount, pt->device), "SM count");
    spmvk::build_plan(pt, n, row_ptr, col_idx, vals);
    spmvk::build_tiles(pt, spmvk::default_tile_geom());
    build_dag(pt);
    *out = pt;
    pt = nullptr;
    return SPMV_OK;
    }
    catch (const spmvk::Fail& f) {
        if (pt) { spmvk::free_plan(pt); delete pt; }
        return fail_status(f.code, f.msg);
    }
    catch (const std::bad_alloc&) {
        if (pt) { spmvk::free_plan(pt); delete pt; }
        return fail_status(SPMV_ENOMEM, "host allocation failed");
    }
    catch (...) {
        if (pt) { spmvk::free_plan(pt); delete pt; }
        return fail_status(SPMV_EINVAL, "unexpected exception");
    }
}

int spmv_part_destroy(spmv_part* pt) {
    if (!pt) return SPMV_OK;
    cudaError_t e = cudaDeviceSynchronize();
    spmvk::free_plan(pt);
    delete pt;
    if (e != cudaSuccess) return fail_status(SPMV_ECUDA, cudaGetErrorString(e));
    return SPMV_OK;
}

int spmv_part_query(const spmv_part* pt, int what, int part_idx, int64_t* out) {
    API_TRY
    check_part(pt);
    need(out != nullptr, SPMV_EINVAL, "out is NULL");
    switch (what) {
        case SPMV_Q_N: *out = pt->n; break;
        case SPMV_Q_P: *out = pt->P; break;
        case SPMV_Q_GRANULARITY: *out = pt->gran; break;
        case SPMV_Q_NNZ: *out = pt->nnz; break;
        case SPMV_Q_NNZ_LOCAL: *out = pt->nnz_l; break;
        case SPMV_Q_NNZ_REMOTE: *out = pt->nnz_r; break;
        case SPMV_Q_N_SEND: *out = pt->n_send; break;
        case SPMV_Q_N_HALO:
            if (part_idx < 0 || part_idx >= pt->P) fail(SPMV_EINVAL, "rank %d", part_idx);
            *out = pt->halo_off[part_idx + 1] - pt->halo_off[part_idx];
            break;
        case SPMV_Q_N_REMOTE_ROWS: *out = pt->n_rr; break;
        case SPMV_Q_N_OPS: *out = pt->n_ops; break;
        case SPMV_Q_N_EDGES: *out = (int64_t)pt->edges.size(); break;
        case SPMV_Q_ALG_BYTES: *out = alg_bytes_total(pt); break;
        case SPMV_Q_ALG_BYTES_LOCAL: *out = alg_bytes_local(pt); break;
        case SPMV_Q_DEVICE_BYTES: *out = (int64_t)pt->device_bytes; break;
        case SPMV_Q_LAST_RECORDS: *out = pt->last_records; break;
        case SPMV_Q_LAST_WAITS: *out = pt->last_waits; break;
        case SPMV_Q_ERROR: {
            int h = 0;
            check_cuda(cudaDeviceSynchronize(), "synchronize");
            check_cuda(cudaMemcpy(&h, pt->err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
            *out = h;
            break;
        }
        case SPMV_Q_LOCAL_VARIANT: *out = pt->variant[0] * 100 + pt->vparam[0]; break;
        case SPMV_Q_REMOTE_VARIANT: *out = pt->variant[1] * 100 + pt->vparam[1]; break;
        case SPMV_Q_SELL_ENTRIES: *out = pt->sell_entries; break;
        case SPMV_Q_N_LOCAL_TILES: *out = pt->ltile_off.empty() ? 0 : pt->ltile_off[pt->P]; break;
        case SPMV_Q_LAST_LAUNCHES: *out = pt->last_launches; break;
        case SPMV_Q_LAST_DEFERRED: *out = pt->last_deferred; break;
        default: fail(SPMV_EINVAL, "unknown query %d", what);
    }
    API_CATCH
    return SPMV_OK;
}

int64_t spmv_part_export_len(const spmv_part* pt, int what, int p) {
    if (!pt) return -1;
    const bool rank_ok = p >= 0 && p < pt->P;
    const int64_t rows = rank_ok ? pt->bounds[p + 1] - pt->bounds[p] : 0;
    switch (what) {
        case SPMV_X_BOUNDS: return pt->P + 1;
        case SPMV_X_SEND_IDX: return pt->n_send;
        case SPMV_X_HALO_OFF: return pt->P + 1;
        case SPMV_X_SEG_OFF: return (int64_t)pt->P * pt->P + 1;
        case SPMV_X_SENDBUF: return pt->n_send;
        case SPMV_X_RECVBUF: return pt->n_send;
        default: break;
    }
    if (!rank_ok) return -1;
    switch (what) {
        case SPMV_X_L_PTR: return rows + 1;
        case SPMV_X_R_PTR: return rows + 1;
        case SPMV_X_HALO: return pt->halo_off[p + 1] - pt->halo_off[p];
        case SPMV_X_L_COL:
        case SPMV_X_L_VAL: {
            int32_t a = 0, b = 0;
            if (cudaMemcpy(&a, pt->l_ptr + pt->bounds[p], 4, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            if (cudaMemcpy(&b, pt->l_ptr + pt->bounds[p + 1], 4, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            return (int64_t)b - a;
        }
        case SPMV_X_R_COL:
        case SPMV_X_R_VAL: {
            int32_t a = 0, b = 0;
            if (cudaMemcpy(&a, pt->rr_ptr + pt->rr_off[p], 4, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            if (cudaMemcpy(&b, pt->rr_ptr + pt->rr_off[p + 1], 4, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            return (int64_t)b - a;
        }
        default: return -1;
    }
}

int spmv_part_export_plan(const spmv_part* pt, int what, int p, void* dst, int64_t cap) {
    API_TRY
    check_part(pt);
    const int64_t len = spmv_part_export_len(pt, what, p);
    if (len < 0) fail(SPMV_EINVAL, "bad selector %d / rank %d", what, p);
    if (len > cap) fail(SPMV_EINVAL, "capacity %lld < %lld", (long long)cap, (long long)len);
    if (len > 0 && !dst) fail(SPMV_EINVAL, "host_dst is NULL");
    if (len == 0) return SPMV_OK;
    check_cuda(cudaDeviceSynchronize(), "synchronize");
    if (what == SPMV_X_L_COL || what == SPMV_X_L_VAL || what == SPMV_X_R_COL || what == SPMV_X_R_VAL)
        spmvk::restore_csr(const_cast<spmv_part*>(pt));   // the matrix is unchanged; its CSR copy is rebuilt
    int64_t* d64 = static_cast<int64_t*>(dst);
    int32_t* d32 = static_cast<int32_t*>(dst);
    double* df = static_cast<double*>(dst);
    switch (what) {
        case SPMV_X_BOUNDS: std::copy(pt->bounds.begin(), pt->bounds.end(), d64); break;
        case SPMV_X_HALO_OFF: std::copy(pt->halo_off.begin(), pt->halo_off.end(), d64); break;
        case SPMV_X_SEG_OFF: std::copy(pt->seg_off.begin(), pt->seg_off.end(), d64); break;
        case SPMV_X_SEND_IDX: {
            auto h = d2h(pt->send_idx, len);
            std::copy(h.begin(), h.end(), d32);
            break;
        }
        case SPMV_X_SENDBUF: {
            auto h = d2h(pt->sendbuf, len);
            std::copy(h.begin(), h.end(), df);
            break;
        }
        case SPMV_X_RECVBUF: {
            auto h = d2h(pt->recvbuf, len);
            std::copy(h.begin(), h.end(), df);
            break;
        }
        case SPMV_X_HALO: {
            auto h = d2h(pt->send_idx + pt->halo_off[p], len);
            std::copy(h.begin(), h.end(), d32);
            break;
        }
        case SPMV_X_L_PTR:
        case SPMV_X_L_COL:
        case SPMV_X_L_VAL: {
            const int64_t rows = pt->bounds[p + 1] - pt->bounds[p];
            auto ptr = d2h(pt->l_ptr + pt->bounds[p], rows + 1);
            if (what == SPMV_X_L_PTR) {
                for (int64_t i = 0; i <= rows; ++i) d64[i] = (int64_t)ptr[(size_t)i] - ptr[0];
            } else if (what == SPMV_X_L_COL) {
                auto h = d2h(pt->l_col + ptr[0], len);
                std::copy(h.begin(), h.end(), d32);
            } else {
                auto h = d2h(pt->l_val + ptr[0], len);
                std::copy(h.begin(), h.end(), df);
            }
            break;
        }
        case SPMV_X_R_PTR: {
            const int64_t rows = pt->bounds[p + 1] - pt->bounds[p];
            const int64_t a = pt->rr_off[p], b = pt->rr_off[p + 1];
            auto rrow = d2h(pt->rr_row + a, b - a);
            auto rptr = d2h(pt->rr_ptr + a, b - a + 1);
            std::vector<int64_t> cnt((size_t)rows + 1, 0);
            for (int64_t i = 0; i < b - a; ++i)
                cnt[(size_t)(rrow[(size_t)i] - pt->bounds[p]) + 1] = (int64_t)rptr[(size_t)i + 1] - rptr[(size_t)i];
            d64[0] = 0;
            for (int64_t i = 1; i <= rows; ++i) d64[i] = d64[i - 1] + cnt[(size_t)i];
            break;
        }
        case SPMV_X_R_COL:
        case SPMV_X_R_VAL: {
            int32_t k0 = 0;
            check_cuda(cudaMemcpy(&k0, pt->rr_ptr + pt->rr_off[p], 4, cudaMemcpyDeviceToHost), "export");
            if (what == SPMV_X_R_COL) {
                auto h = d2h(pt->r_col + k0, len);
                for (int64_t i = 0; i < len; ++i) d32[i] = h[(size_t)i] - (int32_t)pt->halo_off[p];
            } else {
                auto h = d2h(pt->r_val + k0, len);
                std::copy(h.begin(), h.end(), df);
            }
            break;
        }
        default: fail(SPMV_EINVAL, "bad selector %d", what);
    }
    API_CATCH
    return SPMV_OK;
}

int spmv_part_op_info(const spmv_part* pt, int op, int32_t* kind, int32_t* dst, int32_t* src) {
    API_TRY
    check_part(pt);
    need(kind && dst && src, SPMV_EINVAL, "output pointer is NULL");
    if (op < 0 || op >= pt->n_ops) fail(SPMV_EINVAL, "op %d not in [0, %d)", op, pt->n_ops);
    *dst = -1;
    *src = -1;
    if (pt->gran == SPMV_COARSE) {
        *kind = op;
    } else if (pt->gran == SPMV_PER_PARTITION) {
        *kind = op % 4;
        if (*kind == SPMV_OP_PACK) *src = op / 4;
        else *dst = op / 4;
    } else if (op < 2 * pt->P) {
        *kind = op % 2 == 0 ? SPMV_OP_LOCAL : SPMV_OP_REMOTE;
        *dst = op / 2;
    } else {
        const spmv_part::Seg& g = pt->segs[(size_t)(op - 2 * pt->P) / 2];
        *kind = (op - 2 * pt->P) % 2 == 0 ? SPMV_OP_PACK : SPMV_OP_COPY;
        *dst = g.p;
        *src = g.q;
    }
    API_CATCH
    return SPMV_OK;
}

int spmv_part_dag(const spmv_part* pt, int32_t* edges, int64_t cap_pairs, int64_t* n_pairs) {
    API_TRY
    check_part(pt);
    need(n_pairs != nullptr, SPMV_EINVAL, "n_pairs_out is NULL");
    *n_pairs = (int64_t)pt->edges.size();
    if (edges) {
        if (cap_pairs < (int64_t)pt->edges.size()) fail(SPMV_EINVAL, "capacity too small");
        for (size_t i = 0; i < pt->edges.size(); ++i) {
            edges[2 * i] = pt->edges[i].first;
            edges[2 * i + 1] = pt->edges[i].second;
        }
    }
    API_CATCH
    return SPMV_OK;
}

// Validates (variant, param) and prepares the tables it needs.
static void prepare_variant(spmv_part* pt, int variant, int param, int op_kind) {
    if (!pt->graphs.empty()) fail(SPMV_EINVAL, "destroy the captured graphs before changing the variant");
    // every variant but the sliced ones reads the CSR; the 32-bit sliced
    // LOCAL product reads the 32-bit slot columns
    if (pt->csr_released && (variant != SPMV_VARIANT_SELL16 || op_kind != SPMV_OP_LOCAL) &&
        (variant != SPMV_VARIANT_SELL || (op_kind != SPMV_OP_REMOTE && !pt->sell[0].col)))
        spmvk::restore_csr(pt);
    if (variant == SPMV_VARIANT_TILE) {
        static const spmvk::TileGeom geoms[] = {{256, 3456, 2, 16, 2},
                                                {512, 6912, 2, 16, 2},
                                                {256, 3456, 3, 16, 2},
                                                {128, 3456, 2, 32, 1},
                                                {256, 2048, 3, 8, 2}};
        const int ng = (int)(sizeof geoms / sizeof geoms[0]);
        if (param < 0 || param >= ng) fail(SPMV_EINVAL, "tile geometry %d not in [0, %d)", param, ng);
        const spmvk::TileGeom g = geoms[param];
        if (!spmvk::tile_geom_supported(g)) fail(SPMV_EINVAL, "tile geometry not compiled");
        check_cuda(cudaDeviceSynchronize(), "synchronize");
        if (g.rows() != pt->geom.rows() || g.nnz_cap != pt->geom.nnz_cap)
            spmvk::build_tiles(pt, g);
        pt->geom = g;
    } else if (variant == SPMV_VARIANT_VECTOR) {
        if (param != 2 && param != 4 && param != 8 && param != 16 && param != 32)
            fail(SPMV_EINVAL, "vector width %d not in {2,4,8,16,32}", param);
    } else if (variant == SPMV_VARIANT_PAIRS) {
        if (param != 1 && param != 2 && param != 4 && param != 8 && param != 102 && param != 104)
            fail(SPMV_EINVAL, "pair variant %d not in {1,2,4,8,102,104}", param);
    } else if (variant == SPMV_VARIANT_WARP) {
        const int cap = spmvk::warp_tile_cap(param);
        if (cap < 0) fail(SPMV_EINVAL, "warp geometry %d not in [0, 5)", param);
        check_cuda(cudaDeviceSynchronize(), "synchronize");
        if (!pt->lwtiles || pt->wtile_cap != cap) spmvk::build_warp_tiles(pt, cap);
    } else if (variant == SPMV_VARIANT_MERGE) {
        check_cuda(cudaDeviceSynchronize(), "synchronize");
        if (!pt->lmtiles) spmvk::build_merge_tiles(pt);
    } else if (variant == SPMV_VARIANT_SELL || variant == SPMV_VARIANT_SELL16) {
        if (!spmvk::sell_param_supported(param))
            fail(SPMV_EINVAL, "sliced variant %d not in {4,8,9,104..107} (+2000 balanced)", param);
        if (variant == SPMV_VARIANT_SELL16 && op_kind != SPMV_OP_LOCAL)
            fail(SPMV_EINVAL, "16-bit column deltas serve the LOCAL product only");
        check_cuda(cudaDeviceSynchronize(), "synchronize");
        if (!pt->sell_built) spmvk::build_sell(pt);
        if (variant == SPMV_VARIANT_SELL16 && !spmvk::build_sell_delta16(pt))
            fail(SPMV_EINVAL, "a LOCAL column lies more than 32767 rows from its row: no 16-bit deltas");
        if (spmvk::sell_param_balanced(param)) {
            if (op_kind != SPMV_OP_REMOTE) spmvk::build_sell_split(pt, 0, param);
            if (op_kind != SPMV_OP_LOCAL) spmvk::build_sell_split(pt, 1, param);
        }
    } else {
        fail(SPMV_EINVAL, "unknown variant %d", variant);
    }
}

int spmv_part_set_variant(spmv_part* pt, int variant, int param) {
    API_TRY
    check_part(pt);
    if (variant == SPMV_VARIANT_SELL16)
        fail(SPMV_EINVAL, "16-bit column deltas serve the LOCAL product only: use spmv_part_set_op_variant");
    prepare_variant(pt, variant, param, -1);
    pt->variant[0] = pt->variant[1] = variant;
    pt->vparam[0] = pt->vparam[1] = param;
    API_CATCH
    return SPMV_OK;
}

int spmv_part_set_op_variant(spmv_part* pt, int op_kind, int variant, int param) {
    API_TRY
    check_part(pt);
    if (op_kind != SPMV_OP_LOCAL && op_kind != SPMV_OP_REMOTE)
        fail(SPMV_EINVAL, "op kind %d has no product variant", op_kind);
    prepare_variant(pt, variant, param, op_kind);
    const int i = op_kind == SPMV_OP_REMOTE ? 1 : 0;
    pt->variant[i] = variant;
    pt->vparam[i] = param;
    API_CATCH
    return SPMV_OK;
}

int spmv_pack(spmv_part* pt, int p, const double* x, cudaStream_t s) {
    API_TRY
    check_part(pt);
    check_rank(pt, p);
    need(x != nullptr || pt->n == 0, SPMV_EINVAL, "x_dev is NULL");
    pt->last_launches = op_pack(pt, p, x, s);
    API_CATCH
    return SPMV_OK;
}

int spmv_local(spmv_part* pt, int p, const double* x, double* y, cudaStream_t s) {
    API_TRY
    check_part(pt);
    check_rank(pt, p);
    need((x != nullptr && y != nullptr) || pt->n == 0, SPMV_EINVAL, "x_dev or y_dev is NULL");
    pt->last_launches = op_local(pt, p, x, y, s);
    API_CATCH
    return SPMV_OK;
}

int spmv_halo_copy(spmv_part* pt, int p, cudaStream_t s) {
    API_TRY
    check_part(pt);
    check_rank(pt, p);
    pt->last_launches = op_copy(pt, p, s);
    API_CATCH
    return SPMV_OK;
}

int spmv_remote(spmv_part* pt, int p, double* y, cudaStream_t s) {
    API_TRY
    check_part(pt);
    check_rank(pt, p);
    need(y != nullptr || pt->n == 0, SPMV_EINVAL, "y_dev is NULL");
    pt->last_launches = op_remote(pt, p, y, s);
    API_CATCH
    return SPMV_OK;
}

int spmv_schedule_run(spmv_part* pt, const int32_t* order, const int32_t* stream_of, int n_ops,
                      cudaStream_t* streams, int n_streams, const double* x, double* y, int flags,
                      int64_t* handle) {
    API_TRY
    check_part(pt);
    need(streams != nullptr, SPMV_EINVAL, "streams is NULL");
    const bool relaxed = (flags & SPMV_RUN_RELAXED) != 0;
    const bool defer = (flags & SPMV_RUN_DEFER) != 0;
    flags &= ~(SPMV_RUN_RELAXED | SPMV_RUN_DEFER);
    if (flags == SPMV_RUN_REPLAY) {
        need(handle != nullptr, SPMV_EINVAL, "graph handle is NULL");
        auto it = pt->graphs.find(*handle);
        if (it == pt->graphs.end()) fail(SPMV_EINVAL, "unknown graph handle %lld", (long long)*handle);
        if (it->second.x != x || it->second.y != y) fail(SPMV_EINVAL, "x_dev / y_dev differ from the captured ones");
        check_cuda(cudaGraphLaunch(it->second.exec, streams[0]), "cudaGraphLaunch");
        return SPMV_OK;
    }
    if (flags != SPMV_RUN_EAGER && flags != SPMV_RUN_CAPTURE) fail(SPMV_EINVAL, "unknown flags %d", flags);
    if (relaxed && flags != SPMV_RUN_CAPTURE) fail(SPMV_EINVAL, "SPMV_RUN_RELAXED applies to SPMV_RUN_CAPTURE only");
    if (defer && flags != SPMV_RUN_CAPTURE) fail(SPMV_EINVAL, "SPMV_RUN_DEFER applies to SPMV_RUN_CAPTURE only");
    validate_schedule(pt, order, stream_of, n_ops, n_streams);
    need((x != nullptr && y != nullptr) || pt->n == 0, SPMV_EINVAL, "x_dev or y_dev is NULL");
    ensure_events(pt, n_streams);
    if (flags == SPMV_RUN_EAGER) {
        issue(pt, order, stream_of, n_ops, streams, n_streams, x, y, relaxed, defer);
        return SPMV_OK;
    }
    need(handle != nullptr, SPMV_EINVAL, "graph handle is NULL");
    check_cuda(cudaStreamBeginCapture(streams[0], cudaStreamCaptureModeThreadLocal), "begin capture");
    try {
        issue(pt, order, stream_of, n_ops, streams, n_streams, x, y, relaxed, defer);
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(streams[0], &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    cudaGraph_t g = nullptr;
    check_cuda(cudaStreamEndCapture(streams[0], &g), "end capture");
    try {
        fix_deferred_edges(pt, g);
    } catch (...) {
        pt->deferred_nodes.clear();
        cudaGraphDestroy(g);
        throw;
    }
    pt->deferred_nodes.clear();
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    check_cuda(e, "cudaGraphInstantiate");
    const int64_t id = pt->next_graph++;
    pt->graphs[id] = spmvk::GraphRec{exec, x, y};
    *handle = id;
    API_CATCH
    return SPMV_OK;
}

int spmv_graph_destroy(spmv_part* pt, int64_t handle) {
    API_TRY
    check_part(pt);
    auto it = pt->graphs.find(handle);
    if (it == pt->graphs.end()) fail(SPMV_EINVAL, "unknown graph handle %lld", (long long)handle);
    check_cuda(cudaDeviceSynchronize(), "synchronize");
    cudaGraphExecDestroy(it->second.exec);
    pt->graphs.erase(it);
    API_CATCH
    return SPMV_OK;
}

int spmv_part_io_buffers(spmv_part* pt, double** x_out, double** y_out) {
    API_TRY
    check_part(pt);
    need(x_out && y_out, SPMV_EINVAL, "output pointer is NULL");
    if (!pt->io_x) {
        pt->io_x = static_cast<double*>(spmvk::dev_alloc(pt, (size_t)pt->n * sizeof(double)));
        pt->io_y = static_cast<double*>(spmvk::dev_alloc(pt, (size_t)pt->n * sizeof(double)));
    }
    *x_out = pt->io_x;
    *y_out = pt->io_y;
    API_CATCH
    return SPMV_OK;
}

namespace {

// The host path's streams, events and per-rank remote-free runs, made once
// per plan.  Events: 3P+1 used within one product (x block p arrived; LOCAL
// p done; REMOTE p done; exchange done), then per device buffer pair s of
// the streamed path: x_s free (its readers are done), y_s free (its copies
// out are done).
void host_path_setup(spmv_part* pt) {
    const int P = pt->P;
    if (!pt->io_x) {
        pt->io_x = static_cast<double*>(spmvk::dev_alloc(pt, (size_t)pt->n * sizeof(double)));
        pt->io_y = static_cast<double*>(spmvk::dev_alloc(pt, (size_t)pt->n * sizeof(double)));
    }
    while ((int)pt->io_ev.size() < 3 * P + 5) {
        cudaEvent_t e;
        check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        pt->io_ev.push_back(e);
    }
    if (!pt->io_out) check_cuda(cudaStreamCreateWithFlags(&pt->io_out, cudaStreamNonBlocking), "stream");
    if (!pt->io_alt) check_cuda(cudaStreamCreateWithFlags(&pt->io_alt, cudaStreamNonBlocking), "stream");
    if (!pt->io_aux) check_cuda(cudaStreamCreateWithFlags(&pt->io_aux, cudaStreamNonBlocking), "stream");
    if (pt->io_free.empty()) {   // once per plan: the remote-free run of every rank
        std::vector<int32_t> rr((size_t)pt->n_rr);
        if (pt->n_rr)
            check_cuda(cudaMemcpy(rr.data(), pt->rr_row, rr.size() * 4, cudaMemcpyDeviceToHost), "remote rows");
        for (int p = 0; p < P; ++p) {
            int64_t prev = pt->bounds[p], best_a = prev, best_b = prev;
            for (int64_t k = pt->rr_off[p]; k <= pt->rr_off[p + 1]; ++k) {
                const int64_t next = k < pt->rr_off[p + 1] ? (int64_t)rr[(size_t)k] : pt->bounds[p + 1];
                if (next - prev > best_b - best_a) {
                    best_a = prev;
                    best_b = next;
                }
                prev = next + 1;
            }
            pt->io_free.push_back({best_a, best_b});
        }
    }
}

// One product y_host = A x_host through the device vectors xd / yd,
// transfers overlapped with the products (the order is described at
// spmv_apply_host_pipelined).  Nothing waits on the host.  With slot >= 0
// the product is one of a stream of products on two pairs of device vectors:
// its copies in wait until the readers of the same pair's previous x are
// done, its products until the same pair's previous y has gone out, and its
// exchange until the previous product's REMOTE products have read the
// receive buffer (the only other buffers products share).
//   x_blocks: x goes in rank block by rank block (else in one copy, after
//   which every LOCAL product may start); y_parts: each rank's rows go out as
//   soon as they are final (else y goes out in one copy after the last
//   REMOTE product).  A copy costs a few microseconds beyond its bytes, so
//   fewer, larger copies suit a stream of products, where the next
//   product's transfers hide the latency that the pieces shorten.
int64_t host_product(spmv_part* pt, const double* x_host, double* y_host, double* xd, double* yd,
                     cudaStream_t copy_stream, cudaStream_t compute_stream, int slot, bool x_blocks,
                     bool y_parts) {
    const int P = pt->P;
    cudaStream_t out_stream = pt->io_out;
    cudaEvent_t* ev = pt->io_ev.data();
    cudaEvent_t x_free = slot >= 0 ? ev[3 * P + 1 + slot] : nullptr;
    cudaEvent_t y_free = slot >= 0 ? ev[3 * P + 3 + slot] : nullptr;
    // x block by block on the copy stream; rank p's LOCAL product starts as
    // soon as its block has arrived (it reads no other x).  Every copy in is
    // issued before any wait on another stream, so that streams sharing a
    // hardware queue never hold a copy behind a wait.
    int64_t launches = 0;
    if (x_free) check_cuda(cudaStreamWaitEvent(copy_stream, x_free, 0), "wait");
    if (x_blocks) {
        for (int p = 0; p < P; ++p) {
            const int64_t r0 = pt->bounds[p], r1 = pt->bounds[p + 1];
            if (r1 > r0)
                check_cuda(cudaMemcpyAsync(xd + r0, x_host + r0, (size_t)(r1 - r0) * sizeof(double),
                                           cudaMemcpyHostToDevice, copy_stream),
                           "copy x in");
            check_cuda(cudaEventRecord(ev[p], copy_stream), "event");
        }
    } else {
        check_cuda(cudaMemcpyAsync(xd, x_host, (size_t)pt->n * sizeof(double), cudaMemcpyHostToDevice,
                                   copy_stream),
                   "copy x in");
        check_cuda(cudaEventRecord(ev[P - 1], copy_stream), "event");
    }
    auto x_arrived = [&](int p) { return ev[x_blocks ? p : P - 1]; };
    // y goes out on a stream of its own, so that it overlaps the copies in.
    // Each copy out is issued right after the product that finishes its rows,
    // so that it is queued before the host is through issuing the rest.
    auto copy_out = [&](int64_t a, int64_t b) {
        if (b > a && y_parts)
            check_cuda(cudaMemcpyAsync(y_host + a, yd + a, (size_t)(b - a) * sizeof(double),
                                       cudaMemcpyDeviceToHost, out_stream),
                       "copy y out");
    };
    if (y_free) {
        check_cuda(cudaStreamWaitEvent(compute_stream, y_free, 0), "wait");
        check_cuda(cudaStreamWaitEvent(pt->io_alt, y_free, 0), "wait");
    }
    // The LOCAL products (and later the REMOTE products) alternate between
    // compute_stream and a second stream, so that one rank's launch fills the
    // SMs the previous one leaves idle at its tail.  A rank's remote-free run
    // is final after its LOCAL product.
    for (int p = 0; p < P; ++p) {
        cudaStream_t cs = (p & 1) ? pt->io_alt : compute_stream;
        check_cuda(cudaStreamWaitEvent(cs, x_arrived(p), 0), "wait");
        launches += op_local(pt, p, xd, yd, cs);
        check_cuda(cudaEventRecord(ev[P + p], cs), "event");
        if (y_parts) {
            check_cuda(cudaStreamWaitEvent(out_stream, ev[P + p], 0), "wait");
            copy_out(pt->io_free[p].first, pt->io_free[p].second);
        }
    }
    // pack and exchange need all of x: on a third stream as soon as the last
    // block has arrived, beside the LOCAL products.  In a stream of products
    // the exchange first waits for the previous product's REMOTE products
    // (the events still hold their last records).
    check_cuda(cudaStreamWaitEvent(pt->io_aux, ev[P - 1], 0), "wait");
    launches += op_pack(pt, -1, xd, pt->io_aux);
    if (slot >= 0)
        for (int p = 0; p < P; ++p) check_cuda(cudaStreamWaitEvent(pt->io_aux, ev[2 * P + p], 0), "wait");
    launches += op_copy(pt, -1, pt->io_aux);
    check_cuda(cudaEventRecord(ev[3 * P], pt->io_aux), "event");
    if (x_free) {   // x_s is free once the pack and every LOCAL product are done
        for (int p = 0; p < P; ++p) check_cuda(cudaStreamWaitEvent(pt->io_aux, ev[P + p], 0), "wait");
        check_cuda(cudaEventRecord(x_free, pt->io_aux), "event");
    }
    // the remote products rank by rank, each after its own LOCAL product (on
    // the same stream) and the exchange; a rank's other rows go out after its
    // REMOTE product, while the later ranks' products run
    for (int p = 0; p < P; ++p) {
        cudaStream_t cs = (p & 1) ? pt->io_alt : compute_stream;
        check_cuda(cudaStreamWaitEvent(cs, ev[3 * P], 0), "wait");
        launches += op_remote(pt, p, yd, cs);
        check_cuda(cudaEventRecord(ev[2 * P + p], cs), "event");
        check_cuda(cudaStreamWaitEvent(out_stream, ev[2 * P + p], 0), "wait");
        copy_out(pt->bounds[p], pt->io_free[p].first);
        copy_out(pt->io_free[p].second, pt->bounds[p + 1]);
    }
    if (!y_parts)   // every rank's REMOTE product (after its LOCAL one) is done
        check_cuda(cudaMemcpyAsync(y_host, yd, (size_t)pt->n * sizeof(double), cudaMemcpyDeviceToHost,
                                   out_stream),
                   "copy y out");
    if (y_free) check_cuda(cudaEventRecord(y_free, out_stream), "event");
    return launches;
}

}  // namespace

int spmv_apply_host_pipelined(spmv_part* pt, const double* x_host, double* y_host, cudaStream_t copy_stream,
                              cudaStream_t compute_stream) {
    API_TRY
    check_part(pt);
    need(pt->n == 0 || (x_host && y_host), SPMV_EINVAL, "host buffer is NULL");
    need(copy_stream != compute_stream, SPMV_EINVAL, "the copy and compute streams must differ");
    if (pt->n == 0) return SPMV_OK;
    host_path_setup(pt);
    const int64_t launches =
        host_product(pt, x_host, y_host, pt->io_x, pt->io_y, copy_stream, compute_stream, -1, true, true);
    check_cuda(cudaStreamSynchronize(pt->io_out), "synchronize");   // after every REMOTE, so after all work
    check_cuda(cudaStreamSynchronize(copy_stream), "synchronize");
    pt->last_launches = launches;
    API_CATCH
    return SPMV_OK;
}

int spmv_apply_host_many(spmv_part* pt, int64_t count, const double* x_host, int64_t x_stride, double* y_host,
                         int64_t y_stride, int flags, cudaStream_t copy_stream, cudaStream_t compute_stream) {
    API_TRY
    check_part(pt);
    if (flags & ~(SPMV_HOST_X_BLOCKS | SPMV_HOST_Y_PARTS)) fail(SPMV_EINVAL, "unknown flags %d", flags);
    if (count < 0) fail(SPMV_EINVAL, "count = %lld < 0", (long long)count);
    need(x_stride >= 0 && y_stride >= 0, SPMV_EINVAL, "negative stride");
    need(pt->n == 0 || count == 0 || (x_host && y_host), SPMV_EINVAL, "host buffer is NULL");
    need(copy_stream != compute_stream, SPMV_EINVAL, "the copy and compute streams must differ");
    if (count >= 2 && y_stride != 0 && y_stride < pt->n)
        fail(SPMV_EINVAL, "y_stride %lld overlaps the results of consecutive products", (long long)y_stride);
    if (pt->n == 0 || count == 0) return SPMV_OK;
    host_path_setup(pt);
    if (!pt->io_x2) {
        pt->io_x2 = static_cast<double*>(spmvk::dev_alloc(pt, (size_t)pt->n * sizeof(double)));
        pt->io_y2 = static_cast<double*>(spmvk::dev_alloc(pt, (size_t)pt->n * sizeof(double)));
    }
    int64_t launches = 0;
    for (int64_t k = 0; k < count; ++k) {
        const int slot = (int)(k & 1);
        launches += host_product(pt, x_host + k * x_stride, y_host + k * y_stride, slot ? pt->io_x2 : pt->io_x,
                                 slot ? pt->io_y2 : pt->io_y, copy_stream, compute_stream, slot,
                                 (flags & SPMV_HOST_X_BLOCKS) != 0, (flags & SPMV_HOST_Y_PARTS) != 0);
    }
    check_cuda(cudaStreamSynchronize(pt->io_out), "synchronize");   // after every REMOTE, so after all work
    check_cuda(cudaStreamSynchronize(pt->io_aux), "synchronize");
    check_cuda(cudaStreamSynchronize(copy_stream), "synchronize");
    pt->last_launches = launches;
    API_CATCH
    return SPMV_OK;
}

int spmv_apply_host(spmv_part* pt, int64_t handle, const double* x_host, double* y_host, cudaStream_t s) {
    API_TRY
    check_part(pt);
    need(pt->n == 0 || (x_host && y_host), SPMV_EINVAL, "host buffer is NULL");
    auto it = pt->graphs.find(handle);
    if (it == pt->graphs.end()) fail(SPMV_EINVAL, "unknown graph handle %lld", (long long)handle);
    if (!pt->io_x || it->second.x != pt->io_x || it->second.y != pt->io_y)
        fail(SPMV_EINVAL, "graph was not captured on the plan's io buffers");
    const size_t bytes = (size_t)pt->n * sizeof(double);
    if (bytes) check_cuda(cudaMemcpyAsync(pt->io_x, x_host, bytes, cudaMemcpyHostToDevice, s), "copy x in");
    check_cuda(cudaGraphLaunch(it->second.exec, s), "cudaGraphLaunch");
    if (bytes) check_cuda(cudaMemcpyAsync(y_host, pt->io_y, bytes, cudaMemcpyDeviceToHost, s), "copy y out");
    check_cuda(cudaStreamSynchronize(s), "synchronize");
    API_CATCH
    return SPMV_OK;
}

int spmv_csr_merge(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                   const double* x, double* y, cudaStream_t s) {
    API_TRY
    if (n < 0 || nnz < 0) fail(SPMV_EINVAL, "n = %lld, nnz = %lld", (long long)n, (long long)nnz);
    const int items = spmvk::merge_items_per_tile();
    if (n + nnz >= (int64_t(1) << 31) - items) fail(SPMV_EBOUNDS, "n + nnz too large for int32 merge paths");
    if (n == 0) return SPMV_OK;
    if (!row_ptr || !x || !y || (nnz > 0 && (!col_idx || !vals))) fail(SPMV_EINVAL, "NULL device pointer");
    const uintptr_t mis = reinterpret_cast<uintptr_t>(row_ptr) | reinterpret_cast<uintptr_t>(col_idx) |
                          reinterpret_cast<uintptr_t>(vals) | reinterpret_cast<uintptr_t>(x) |
                          reinterpret_cast<uintptr_t>(y);
    if (mis & 15) fail(SPMV_EINVAL, "device arrays must be 16-byte aligned");
    int dev = 0, sms = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int n_tiles = (int)((n + nnz + items - 1) / items);
    void* scratch = nullptr;
    const size_t tile_bytes = (size_t)n_tiles * sizeof(spmvk::MergeTile);
    check_cuda(cudaMallocAsync(&scratch, tile_bytes + (size_t)n_tiles * sizeof(spmvk::Carry), s), "cudaMallocAsync");
    spmvk::MergeTile* tiles = static_cast<spmvk::MergeTile*>(scratch);
    spmvk::Carry* carries = reinterpret_cast<spmvk::Carry*>(static_cast<char*>(scratch) + tile_bytes);
    spmvk::CsrArgs a{};
    a.ptr = row_ptr;
    a.col = col_idx;
    a.val = vals;
    a.rowmap = nullptr;
    a.x = x;
    a.y = y;
    a.accumulate = 0;
    a.n_rows = (int)n;
    a.nnz_total = (int)nnz;
    a.guarded = 1;
    a.err = nullptr;
    a.abort_tile = g_merge_abort_tile.load();
    cudaError_t e = spmvk::launch_merge_partition(row_ptr, 0, (int)n, 0, tiles, n_tiles, s);
    if (e == cudaSuccess) e = spmvk::launch_merge(a, tiles, 0, n_tiles, carries, sms, s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    check_cuda(e, "merge product");
    check_cuda(ef, "cudaFreeAsync");
    API_CATCH
    return SPMV_OK;
}

int spmv_csr_merge_noalloc(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                           const double* vals, const double* x, double* y, cudaStream_t s) {
    API_TRY
    if (n < 0 || nnz < 0) fail(SPMV_EINVAL, "n = %lld, nnz = %lld", (long long)n, (long long)nnz);
    const int64_t cap = spmvk::noalloc_max_items();
    if (n + nnz > cap)
        fail(SPMV_EBOUNDS, "n + nnz = %lld exceeds the fixed scratch of the no-allocation path (at most %lld)",
             (long long)(n + nnz), (long long)cap);
    if (n == 0) return SPMV_OK;
    if (!row_ptr || !x || !y || (nnz > 0 && (!col_idx || !vals))) fail(SPMV_EINVAL, "NULL device pointer");
    const uintptr_t mis = reinterpret_cast<uintptr_t>(row_ptr) | reinterpret_cast<uintptr_t>(col_idx) |
                          reinterpret_cast<uintptr_t>(vals) | reinterpret_cast<uintptr_t>(x) |
                          reinterpret_cast<uintptr_t>(y);
    if (mis & 15) fail(SPMV_EINVAL, "device arrays must be 16-byte aligned");
    int dev = 0, sms = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    spmvk::CsrArgs a{};
    a.ptr = row_ptr;
    a.col = col_idx;
    a.val = vals;
    a.rowmap = nullptr;
    a.x = x;
    a.y = y;
    a.accumulate = 0;
    a.n_rows = (int)n;
    a.nnz_total = (int)nnz;
    a.guarded = 1;
    a.err = nullptr;
    a.abort_tile = g_merge_abort_tile.load();
    check_cuda(spmvk::launch_merge_noalloc(a, sms, s), "no-allocation merge product");
    API_CATCH
    return SPMV_OK;
}

int spmv_csr_error(int64_t* out) {
    API_TRY
    need(out != nullptr, SPMV_EINVAL, "out is NULL");
    check_cuda(cudaDeviceSynchronize(), "synchronize");
    int h = 0;
    check_cuda(spmvk::read_clear_csr_error(&h), "error word");
    *out = h;
    API_CATCH
    return SPMV_OK;
}

int spmv_part_check(spmv_part* pt, int64_t* bad_out) {
    API_TRY
    check_part(pt);
    need(bad_out != nullptr, SPMV_EINVAL, "bad_out is NULL");
    spmvk::restore_csr(pt);   // the checks read the CSR
    const int P = pt->P;
    // host tables of group offsets and ranges, one device copy
    std::vector<int64_t> tab;
    auto put = [&](const std::vector<int64_t>& v) {
        const size_t at = tab.size();
        tab.insert(tab.end(), v.begin(), v.end());
        return at;
    };
    std::vector<int64_t> zeros(P, 0), bsize(P), blo(P), bhi(P), hlo(P), hhi(P);
    for (int p = 0; p < P; ++p) {
        bsize[p] = pt->bounds[p + 1] - pt->bounds[p];
        blo[p] = pt->bounds[p];
        bhi[p] = pt->bounds[p + 1];
        hlo[p] = pt->halo_off[p];
        hhi[p] = pt->halo_off[p + 1];
    }
    std::vector<int64_t> slo((size_t)P * P), shi((size_t)P * P);
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q) {
            slo[(size_t)p * P + q] = pt->bounds[q];
            shi[(size_t)p * P + q] = pt->bounds[q + 1];
        }
    const size_t t_bounds = put(pt->bounds), t_zero = put(zeros), t_bsize = put(bsize), t_blo = put(blo),
                 t_bhi = put(bhi), t_rr = put(pt->rr_off), t_hlo = put(hlo), t_hhi = put(hhi),
                 t_seg = put(pt->seg_off), t_slo = put(slo), t_shi = put(shi),
                 t_one = put(std::vector<int64_t>{0, pt->n_send});
    int64_t* d_tab = nullptr;
    unsigned long long* d_bad = nullptr;
    check_cuda(cudaMalloc(&d_tab, tab.size() * sizeof(int64_t) + 64), "check tables");
    cudaError_t e = cudaMalloc(&d_bad, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(d_tab);
        check_cuda(e, "check counter");
    }
    auto run = [&]() -> cudaError_t {
        cudaError_t r = cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (r == cudaSuccess) r = cudaMemset(d_bad, 0, sizeof(unsigned long long));
        const int sms = pt->num_sms;
        // A_L: row i of rank p has columns in [0, r_{p+1} - r_p)
        if (r == cudaSuccess)
            r = spmvk::launch_check_csr(pt->l_ptr, pt->l_col, pt->n, pt->nnz_l, d_tab + t_bounds, P,
                                        d_tab + t_zero, d_tab + t_bsize, d_bad, sms, 0);
        // A_R: remote row k of rank p has receive-buffer positions in p's halo
        if (r == cudaSuccess)
            r = spmvk::launch_check_csr(pt->rr_ptr, pt->r_col, pt->n_rr, pt->nnz_r, d_tab + t_rr, P,
                                        d_tab + t_hlo, d_tab + t_hhi, d_bad, sms, 0);
        // remote rows of rank p are p's rows
        if (r == cudaSuccess)
            r = spmvk::launch_check_list(pt->rr_row, pt->n_rr, d_tab + t_rr, P, d_tab + t_blo, d_tab + t_bhi,
                                         d_bad, sms, 0);
        // send slot of segment (dst p, src q) names a row of q
        if (r == cudaSuccess)
            r = spmvk::launch_check_list(pt->send_idx, pt->n_send, d_tab + t_seg, P * P, d_tab + t_slo,
                                         d_tab + t_shi, d_bad, sms, 0);
        if (r == cudaSuccess)
            r = spmvk::launch_check_list(pt->pack_pos, pt->n_send, d_tab + t_one, 1, d_tab + t_one,
                                         d_tab + t_one + 1, d_bad, sms, 0);
        if (r == cudaSuccess && pt->sell_built) {
            for (int part = 0; part < 2 && r == cudaSuccess; ++part) {
                const spmv_part::SellPart& sp = pt->sell[part];
                const int64_t npos = part ? pt->n_rr : pt->n;
                const int64_t xhi = part ? pt->n_send : pt->n;
                const int32_t* cptr = part ? pt->rr_ptr : pt->l_ptr;
                r = spmvk::launch_check_sell(sp.slices, (int)sp.slice_off[P], sp.len, sp.perm, sp.col, nullptr,
                                             sp.entries, npos, 0, xhi, sp.longs, (int)sp.long_off[P], cptr, d_bad,
                                             sms, 0);
                if (r == cudaSuccess && sp.col16)
                    r = spmvk::launch_check_sell(sp.slices, (int)sp.slice_off[P], sp.len, sp.perm, nullptr,
                                                 sp.col16, sp.entries, npos, 0, xhi, sp.longs, 0, cptr, d_bad,
                                                 sms, 0);
                // the composed y rows of rank p's remote positions are p's rows
                if (r == cudaSuccess && sp.ypos)
                    r = spmvk::launch_check_list(sp.ypos, pt->n_rr, d_tab + t_rr, P, d_tab + t_blo, d_tab + t_bhi,
                                                 d_bad, sms, 0);
            }
        }
        unsigned long long h = 0;
        if (r == cudaSuccess) r = cudaDeviceSynchronize();
        if (r == cudaSuccess) r = cudaMemcpy(&h, d_bad, sizeof h, cudaMemcpyDeviceToHost);
        *bad_out = (int64_t)h;
        return r;
    };
    e = run();
    cudaFree(d_tab);
    cudaFree(d_bad);
    check_cuda(e, "index check");
    API_CATCH
    return SPMV_OK;
}

int spmv_selftest_check(int64_t* found_out) {
    API_TRY
    need(found_out != nullptr, SPMV_EINVAL, "found_out is NULL");
    // a 3-row CSR whose column 5 lies outside [0, 4), and an index list
    // whose 7 lies outside [0, 3): the checks must find exactly these two
    const int32_t h_ptr[4] = {0, 2, 3, 3}, h_col[3] = {0, 5, 1}, h_idx[3] = {0, 7, 2};
    const int64_t h_tab[4] = {0, 0, 4, 3};   // offsets {0}, lo {0}, hi {4}; list hi {3}
    int32_t* d_i = nullptr;
    int64_t* d_t = nullptr;
    unsigned long long* d_bad = nullptr;
    check_cuda(cudaMalloc(&d_i, 16 * sizeof(int32_t)), "self-test");
    cudaError_t e = cudaMalloc(&d_t, 4 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(d_i, h_ptr, sizeof h_ptr, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_i + 4, h_col, sizeof h_col, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_i + 8, h_idx, sizeof h_idx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_t, h_tab, sizeof h_tab, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = spmvk::launch_check_csr(d_i, d_i + 4, 3, 3, d_t, 1, d_t + 1, d_t + 2, d_bad, 1, 0);
    if (e == cudaSuccess) e = spmvk::launch_check_list(d_i + 8, 3, d_t, 1, d_t + 1, d_t + 3, d_bad, 1, 0);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_bad, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d_i);
    cudaFree(d_t);
    cudaFree(d_bad);
    check_cuda(e, "self-test");
    *found_out = (int64_t)h;
    API_CATCH
    return SPMV_OK;
}

int spmv_selftest_wait_timeout(int64_t limit_ns, int64_t* status_out) {
    API_TRY
    need(status_out != nullptr, SPMV_EINVAL, "status_out is NULL");
    if (limit_ns < 1000 || limit_ns > 2000000000) fail(SPMV_EINVAL, "limit %lld ns not in [1e3, 2e9]", (long long)limit_ns);
    int st = 0;
    check_cuda(spmvk::selftest_wait_timeout((uint64_t)limit_ns, &st), "self-test");
    *status_out = st;
    API_CATCH
    return SPMV_OK;
}

int spmv_probe_dfma(int64_t iters, int ctas_per_sm, int lanes, double* out_dev, int64_t out_cap,
                    int64_t* dfma_out, cudaStream_t s) {
    API_TRY
    need(out_dev != nullptr && dfma_out != nullptr, SPMV_EINVAL, "NULL pointer");
    if (iters < 1 || iters > (int64_t(1) << 40)) fail(SPMV_EINVAL, "iters = %lld", (long long)iters);
    if (ctas_per_sm < 1 || ctas_per_sm > 8) fail(SPMV_EINVAL, "ctas_per_sm = %d not in [1, 8]", ctas_per_sm);
    if (lanes < 1 || lanes > 32) fail(SPMV_EINVAL, "lanes = %d not in [1, 32]", lanes);
    if (reinterpret_cast<uintptr_t>(out_dev) & 7) fail(SPMV_EINVAL, "out_dev must be 8-byte aligned");
    int dev = 0, sms = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int grid = sms * ctas_per_sm;
    if (out_cap < (int64_t)grid * spmvk::probe_threads())
        fail(SPMV_EINVAL, "out_cap %lld below the %lld threads of the launch", (long long)out_cap,
             (long long)grid * spmvk::probe_threads());
    check_cuda(spmvk::launch_dfma_probe(iters, grid, lanes, out_dev, dfma_out, s), "FP64 probe");
    API_CATCH
    return SPMV_OK;
}

int spmv_probe_gather(const double* table_dev, const int32_t* idx_dev, int64_t count, int ctas_per_sm,
                      double* out_dev, int64_t out_cap, cudaStream_t s) {
    API_TRY
    need(table_dev != nullptr && idx_dev != nullptr && out_dev != nullptr, SPMV_EINVAL, "NULL pointer");
    if (count < 0) fail(SPMV_EINVAL, "count = %lld", (long long)count);
    if (ctas_per_sm < 1 || ctas_per_sm > 8) fail(SPMV_EINVAL, "ctas_per_sm = %d not in [1, 8]", ctas_per_sm);
    if ((reinterpret_cast<uintptr_t>(out_dev) | reinterpret_cast<uintptr_t>(table_dev)) & 7 ||
        reinterpret_cast<uintptr_t>(idx_dev) & 3)
        fail(SPMV_EINVAL, "misaligned pointer");
    int dev = 0, sms = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int grid = sms * ctas_per_sm;
    if (out_cap < (int64_t)grid * spmvk::probe_threads())
        fail(SPMV_EINVAL, "out_cap %lld below the %lld threads of the launch", (long long)out_cap,
             (long long)grid * spmvk::probe_threads());
    check_cuda(spmvk::launch_gather_probe(table_dev, idx_dev, count, grid, out_dev, s), "gather probe");
    API_CATCH
    return SPMV_OK;
}

int spmv_part_release_csr(spmv_part* pt) {
    API_TRY
    check_part(pt);
    if (!pt->graphs.empty()) fail(SPMV_EINVAL, "captured graphs exist (they hold the current arrays)");
    spmvk::release_csr(pt);
    API_CATCH
    return SPMV_OK;
}

int spmv_selftest_merge_abort(int64_t tile) {
    API_TRY
    if (tile < -1 || tile >= (int64_t(1) << 30)) fail(SPMV_EINVAL, "tile %lld not in [-1, 2^30)", (long long)tile);
    g_merge_abort_tile.store((int)(tile + 1));
    API_CATCH
    return SPMV_OK;
}

const char* spmv_last_error(void) { return g_err.c_str(); }

}  // extern "C"
