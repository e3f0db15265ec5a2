"""Python binding of the C ABI in ``include/spmv.h`` (ctypes).

Functions carry the C names and only marshal arguments: device pointers are
ints or objects with ``data_ptr()`` (PyTorch tensors), streams are ints or
objects with ``cuda_stream`` (``torch.cuda.Stream``).  Every step of the
product runs in ``libspmv.so``; there is no fallback: importing this module
fails if the library is not built.
"""
import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspmv.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "spmv.h")

# status codes and selectors (include/spmv.h)
OK, EINVAL, ENOMEM, ECUDA, ESCHED, EBOUNDS, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
OP_PACK, OP_LOCAL, OP_COPY, OP_REMOTE = 0, 1, 2, 3
COARSE, PER_PARTITION, PER_SEGMENT = 0, 1, 2
RUN_EAGER, RUN_CAPTURE, RUN_REPLAY, RUN_RELAXED, RUN_DEFER = 0, 1, 2, 4, 8
HOST_X_BLOCKS, HOST_Y_PARTS = 1, 2
VARIANT_TILE, VARIANT_VECTOR, VARIANT_MERGE, VARIANT_PAIRS, VARIANT_WARP, VARIANT_SELL, VARIANT_SELL16 = (
    0, 1, 2, 3, 4, 5, 6)
SERVE_BATCHED, SERVE_PLAIN = 0, 1
BATCH_SLICED = 64
(Q_N, Q_P, Q_GRANULARITY, Q_NNZ, Q_NNZ_LOCAL, Q_NNZ_REMOTE, Q_N_SEND, Q_N_HALO,
 Q_N_REMOTE_ROWS, Q_N_OPS, Q_N_EDGES, Q_ALG_BYTES, Q_ALG_BYTES_LOCAL,
 Q_DEVICE_BYTES, Q_LAST_RECORDS, Q_LAST_WAITS, Q_ERROR, Q_LOCAL_VARIANT,
 Q_N_LOCAL_TILES, Q_LAST_LAUNCHES, Q_REMOTE_VARIANT, Q_SELL_ENTRIES, Q_LAST_DEFERRED) = range(23)
(BQ_COUNT, BQ_TOTAL_ROWS, BQ_TOTAL_NNZ, BQ_ITEMS, BQ_ALG_BYTES, BQ_OFFSET, BQ_N, BQ_NNZ,
 BQ_LANES, BQ_DEVICE_BYTES, BQ_LAUNCHES) = range(11)
(X_BOUNDS, X_L_PTR, X_L_COL, X_L_VAL, X_R_PTR, X_R_COL, X_R_VAL, X_HALO,
 X_SEND_IDX, X_HALO_OFF, X_SEG_OFF, X_SENDBUF, X_RECVBUF) = range(13)
_X_DTYPE = {X_BOUNDS: np.int64, X_L_PTR: np.int64, X_L_COL: np.int32,
            X_L_VAL: np.float64, X_R_PTR: np.int64, X_R_COL: np.int32,
            X_R_VAL: np.float64, X_HALO: np.int32, X_SEND_IDX: np.int32,
            X_HALO_OFF: np.int64, X_SEG_OFF: np.int64, X_SENDBUF: np.float64,
            X_RECVBUF: np.float64}


class SpmvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("spmv error %d: %s" % (code, msg))
        self.code = code


def declared_functions():
    """Names of the functions include/spmv.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spmv_\w+)\s*\(", text)))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libspmv.so is not built (run __graft_entry__.build() "
                          "or python -m paper_2203_02530_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P64 = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "spmv_part_create": [i64, vp, vp, vp, i32, i32, ctypes.POINTER(vp)],
        "spmv_part_destroy": [vp],
        "spmv_part_query": [vp, i32, i32, P64],
        "spmv_part_export_len": [vp, i32, i32],
        "spmv_part_export_plan": [vp, i32, i32, vp, i64],
        "spmv_part_dag": [vp, vp, i64, P64],
        "spmv_part_op_info": [vp, i32, vp, vp, vp],
        "spmv_part_set_variant": [vp, i32, i32],
        "spmv_part_set_op_variant": [vp, i32, i32, i32],
        "spmv_part_release_csr": [vp],
        "spmv_pack": [vp, i32, vp, vp],
        "spmv_local": [vp, i32, vp, vp, vp],
        "spmv_halo_copy": [vp, i32, vp],
        "spmv_remote": [vp, i32, vp, vp],
        "spmv_schedule_run": [vp, vp, vp, i32, vp, i32, vp, vp, i32, P64],
        "spmv_graph_destroy": [vp, i64],
        "spmv_part_io_buffers": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)],
        "spmv_apply_host": [vp, i64, vp, vp, vp],
        "spmv_apply_host_pipelined": [vp, vp, vp, vp, vp],
        "spmv_apply_host_many": [vp, i64, vp, i64, vp, i64, i32, vp, vp],
        "spmv_csr_merge": [i64, i64, vp, vp, vp, vp, vp, vp],
        "spmv_csr_merge_noalloc": [i64, i64, vp, vp, vp, vp, vp, vp],
        "spmv_csr_error": [P64],
        "spmv_batch_create": [i32, vp, vp, vp, vp, ctypes.POINTER(vp)],
        "spmv_batch_destroy": [vp],
        "spmv_batch_set_lanes": [vp, i32, i32],
        "spmv_batch_query": [vp, i32, i32, P64],
        "spmv_batch_run": [vp, vp, vp, vp],
        "spmv_batch_run_separate": [vp, i32, vp, vp, vp],
        "spmv_batch_release_csr": [vp],
        "spmv_batch_run_host": [vp, vp, vp, i32, vp, vp, vp],
        "spmv_batch_run_host_many": [vp, i64, vp, i64, vp, i64, i32, vp, vp, vp],
        "spmv_serve_create": [vp, i32, i64, ctypes.POINTER(vp)],
        "spmv_serve_destroy": [vp],
        "spmv_serve_run": [vp, i64, vp, vp, vp, vp, i32, vp, vp, vp],
        "spmv_serve_single": [vp, i32, i32, ctypes.c_uint64, vp, vp, vp],
        "spmv_serve_launches": [vp, P64],
        "spmv_serve_set_group_max": [vp, i32],
        "spmv_serve_pm1_bits": [ctypes.c_uint64],
        "spmv_selftest_wait_timeout": [i64, P64],
        "spmv_selftest_merge_abort": [i64],
        "spmv_probe_dfma": [i64, i32, i32, vp, i64, P64, vp],
        "spmv_probe_gather": [vp, vp, i64, i32, vp, i64, vp],
        "spmv_part_check": [vp, P64],
        "spmv_selftest_check": [P64],
        "spmv_last_error": [],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    L.spmv_part_export_len.restype = i64
    L.spmv_serve_pm1_bits.restype = ctypes.c_uint64
    L.spmv_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(a))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def spmv_last_error():
    return lib.spmv_last_error().decode()


def _check(rc):
    if rc != OK:
        raise SpmvError(rc, spmv_last_error())


def spmv_part_create(n, row_ptr, col_idx, vals, P, granularity=COARSE):
    """Build a plan from HOST CSR arrays; returns the opaque handle."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(vals, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib.spmv_part_create(int(n), _ptr(rp), _ptr(ci), _ptr(va), int(P),
                                int(granularity), ctypes.byref(h)))
    return h


def spmv_part_destroy(h):
    _check(lib.spmv_part_destroy(h))


def spmv_part_query(h, what, part_idx=-1):
    out = ctypes.c_int64()
    _check(lib.spmv_part_query(h, int(what), int(part_idx), ctypes.byref(out)))
    return out.value


def spmv_part_export_len(h, what, part_idx=-1):
    return int(lib.spmv_part_export_len(h, int(what), int(part_idx)))


def spmv_part_export_plan(h, what, part_idx=-1):
    n = spmv_part_export_len(h, what, part_idx)
    if n < 0:
        raise SpmvError(EINVAL, "bad export selector")
    out = np.empty(n, dtype=_X_DTYPE[what])
    _check(lib.spmv_part_export_plan(h, int(what), int(part_idx), _ptr(out), n))
    return out


def spmv_part_dag(h):
    n = ctypes.c_int64()
    _check(lib.spmv_part_dag(h, None, 0, ctypes.byref(n)))
    buf = np.empty(2 * n.value, dtype=np.int32)
    _check(lib.spmv_part_dag(h, _ptr(buf), n.value, ctypes.byref(n)))
    return [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(n.value)]


def spmv_part_set_variant(h, variant, param=0):
    _check(lib.spmv_part_set_variant(h, int(variant), int(param)))


def spmv_part_set_op_variant(h, op_kind, variant, param=0):
    _check(lib.spmv_part_set_op_variant(h, int(op_kind), int(variant), int(param)))


def spmv_part_release_csr(h):
    """Free the plan's CSR copy once both products use the sliced layout."""
    _check(lib.spmv_part_release_csr(h))


def spmv_pack(h, part_idx, x_dev, stream):
    _check(lib.spmv_pack(h, int(part_idx), _ptr(x_dev), _stream(stream)))


def spmv_local(h, part_idx, x_dev, y_dev, stream):
    _check(lib.spmv_local(h, int(part_idx), _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def spmv_halo_copy(h, part_idx, stream):
    _check(lib.spmv_halo_copy(h, int(part_idx), _stream(stream)))


def spmv_remote(h, part_idx, y_dev, stream):
    _check(lib.spmv_remote(h, int(part_idx), _ptr(y_dev), _stream(stream)))


def spmv_schedule_run(h, op_order, stream_of_op, streams, x_dev, y_dev,
                      flags=RUN_EAGER, graph_handle=0):
    """Run, capture or replay one implementation; returns the graph handle."""
    order = np.ascontiguousarray(op_order, dtype=np.int32)
    smap = np.ascontiguousarray(stream_of_op, dtype=np.int32)
    sarr = (ctypes.c_void_p * len(streams))(*[_stream(s).value for s in streams])
    g = ctypes.c_int64(int(graph_handle))
    _check(lib.spmv_schedule_run(h, _ptr(order), _ptr(smap), len(order), sarr,
                                 len(streams), _ptr(x_dev), _ptr(y_dev), int(flags),
                                 ctypes.byref(g)))
    return g.value


def spmv_graph_destroy(h, graph_handle):
    _check(lib.spmv_graph_destroy(h, int(graph_handle)))


def spmv_part_io_buffers(h):
    x = ctypes.c_void_p()
    y = ctypes.c_void_p()
    _check(lib.spmv_part_io_buffers(h, ctypes.byref(x), ctypes.byref(y)))
    return x.value, y.value


def spmv_apply_host(h, graph_handle, x_host, y_host, stream):
    _check(lib.spmv_apply_host(h, int(graph_handle), _ptr(x_host), _ptr(y_host),
                               _stream(stream)))


def spmv_apply_host_pipelined(h, x_host, y_host, copy_stream, compute_stream):
    _check(lib.spmv_apply_host_pipelined(h, _ptr(x_host), _ptr(y_host), _stream(copy_stream),
                                         _stream(compute_stream)))


def spmv_apply_host_many(h, count, x_host, x_stride, y_host, y_stride, flags, copy_stream, compute_stream):
    """count independent products through host buffers, consecutive ones
    overlapped (strides in doubles; 0 reuses the same host vector; flags
    HOST_X_BLOCKS / HOST_Y_PARTS choose the copies' granularity)."""
    _check(lib.spmv_apply_host_many(h, int(count), _ptr(x_host), int(x_stride), _ptr(y_host),
                                    int(y_stride), int(flags), _stream(copy_stream), _stream(compute_stream)))


def spmv_csr_merge(n, nnz, row_ptr_dev, col_idx_dev, vals_dev, x_dev, y_dev, stream):
    _check(lib.spmv_csr_merge(int(n), int(nnz), _ptr(row_ptr_dev), _ptr(col_idx_dev),
                              _ptr(vals_dev), _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def spmv_csr_merge_noalloc(n, nnz, row_ptr_dev, col_idx_dev, vals_dev, x_dev, y_dev, stream):
    """spmv_csr_merge with its scratch in the library's fixed device array
    (no allocation during the call; see include/spmv.h for the limit)."""
    _check(lib.spmv_csr_merge_noalloc(int(n), int(nnz), _ptr(row_ptr_dev), _ptr(col_idx_dev),
                                      _ptr(vals_dev), _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def spmv_part_check(h):
    """Indices of the plan outside their ranges (0 for a sound plan)."""
    out = ctypes.c_int64()
    _check(lib.spmv_part_check(h, ctypes.byref(out)))
    return out.value


def spmv_selftest_check():
    out = ctypes.c_int64()
    _check(lib.spmv_selftest_check(ctypes.byref(out)))
    return out.value


def spmv_selftest_wait_timeout(limit_ns):
    out = ctypes.c_int64()
    _check(lib.spmv_selftest_wait_timeout(int(limit_ns), ctypes.byref(out)))
    return out.value


def spmv_probe_dfma(iters, ctas_per_sm, lanes, out_dev, out_cap, stream):
    """Launch the FP64 FMA throughput probe; returns the DFMAs it executes."""
    out = ctypes.c_int64()
    _check(lib.spmv_probe_dfma(int(iters), int(ctas_per_sm), int(lanes), _ptr(out_dev), int(out_cap),
                               ctypes.byref(out), _stream(stream)))
    return out.value


def spmv_probe_gather(table_dev, idx_dev, count, ctas_per_sm, out_dev, out_cap, stream):
    """Launch the gather throughput probe (count gathers)."""
    _check(lib.spmv_probe_gather(_ptr(table_dev), _ptr(idx_dev), int(count), int(ctas_per_sm), _ptr(out_dev),
                                 int(out_cap), _stream(stream)))


def spmv_selftest_merge_abort(tile):
    """Make the plan-free merge launches give up from merge tile `tile` on
    (-1: off); a test hook of the bounded-wait give-up path."""
    _check(lib.spmv_selftest_merge_abort(int(tile)))


def spmv_csr_error():
    out = ctypes.c_int64()
    _check(lib.spmv_csr_error(ctypes.byref(out)))
    return out.value


def spmv_part_op_info(h, op):
    """(kind, destination rank, source rank) of op id `op`; -1 where none."""
    k, d, sr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.spmv_part_op_info(h, int(op), ctypes.byref(k), ctypes.byref(d), ctypes.byref(sr)))
    return k.value, d.value, sr.value


class Part:
    """Owns one plan handle; methods forward to the functions above."""

    def __init__(self, n, row_ptr, col_idx, vals, P, granularity=COARSE):
        self.h = spmv_part_create(n, row_ptr, col_idx, vals, P, granularity)
        self.n, self.P, self.granularity = int(n), int(P), granularity

    def close(self):
        if self.h is not None:
            spmv_part_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def query(self, what, part_idx=-1):
        return spmv_part_query(self.h, what, part_idx)

    def export(self, what, part_idx=-1):
        return spmv_part_export_plan(self.h, what, part_idx)

    def dag(self):
        return spmv_part_dag(self.h)

    def op_names(self):
        """Readable op names: Pack / yL / Copy / yR, with the rank (coarse:
        none; per partition: the rank; per segment: yL2, Pack1to2, ...)."""
        base = {OP_PACK: "Pack", OP_LOCAL: "yL", OP_COPY: "Copy", OP_REMOTE: "yR"}
        out = []
        for op in range(self.n_ops):
            k, d, sr = spmv_part_op_info(self.h, op)
            if d >= 0 and sr >= 0:
                out.append("%s%dto%d" % (base[k], sr, d))
            else:
                r = d if d >= 0 else sr
                out.append(base[k] + ("" if r < 0 else str(r)))
        return out

    @property
    def n_ops(self):
        return self.query(Q_N_OPS)

    def set_variant(self, variant, param=0):
        spmv_part_set_variant(self.h, variant, param)

    def set_op_variant(self, op_kind, variant, param=0):
        spmv_part_set_op_variant(self.h, op_kind, variant, param)

    def release_csr(self):
        spmv_part_release_csr(self.h)

    def run(self, order, stream_of_op, streams, x, y, flags=RUN_EAGER, graph=0):
        return spmv_schedule_run(self.h, order, stream_of_op, streams, x, y, flags, graph)


def spmv_batch_create(mats):
    """mats: list of (n, row_ptr, col_idx, vals) host CSR; returns (handle,
    arrays kept alive until the call returns)."""
    keep = []
    ns = np.array([int(m[0]) for m in mats], dtype=np.int64)
    ptrs = (ctypes.c_void_p * len(mats))()
    cols = (ctypes.c_void_p * len(mats))()
    vals = (ctypes.c_void_p * len(mats))()
    for i, (n, rp, ci, va) in enumerate(mats):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        va = np.ascontiguousarray(va, dtype=np.float64)
        keep += [rp, ci, va]
        ptrs[i] = rp.ctypes.data
        cols[i] = ci.ctypes.data if ci.size else None
        vals[i] = va.ctypes.data if va.size else None
    h = ctypes.c_void_p()
    _check(lib.spmv_batch_create(len(mats), _ptr(ns), ptrs, cols, vals, ctypes.byref(h)))
    return h


def spmv_batch_destroy(h):
    _check(lib.spmv_batch_destroy(h))


def spmv_batch_set_lanes(h, m, lanes):
    _check(lib.spmv_batch_set_lanes(h, int(m), int(lanes)))


def spmv_batch_query(h, what, m=-1):
    out = ctypes.c_int64()
    _check(lib.spmv_batch_query(h, int(what), int(m), ctypes.byref(out)))
    return out.value


def spmv_batch_run(h, x_dev, y_dev, stream):
    _check(lib.spmv_batch_run(h, _ptr(x_dev), _ptr(y_dev), _stream(stream)))


def spmv_batch_run_host(h, x_host, y_host, chunks, s_in, s_compute, s_out):
    _check(lib.spmv_batch_run_host(h, _ptr(x_host), _ptr(y_host), int(chunks), _stream(s_in),
                                   _stream(s_compute), _stream(s_out)))


def spmv_batch_run_host_many(h, count, x_host, x_stride, y_host, y_stride, chunks, s_in, s_compute, s_out):
    """count independent batched products through host buffers, consecutive
    ones overlapped (strides in doubles; 0 reuses the same host vector)."""
    _check(lib.spmv_batch_run_host_many(h, int(count), _ptr(x_host), int(x_stride), _ptr(y_host), int(y_stride),
                                        int(chunks), _stream(s_in), _stream(s_compute), _stream(s_out)))


def spmv_batch_release_csr(h):
    """Keep only the long rows of the batch's CSR once every matrix is sliced."""
    _check(lib.spmv_batch_release_csr(h))


def spmv_batch_run_separate(h, m, x_dev, y_dev, stream):
    _check(lib.spmv_batch_run_separate(h, int(m), _ptr(x_dev), _ptr(y_dev), _stream(stream)))


class Batch:
    """Owns one batch handle (many independent CSR matrices)."""

    def __init__(self, mats):
        self.h = spmv_batch_create(mats)
        self.count = len(mats)

    def close(self):
        if self.h is not None:
            spmv_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def query(self, what, m=-1):
        return spmv_batch_query(self.h, what, m)

    def offsets(self):
        return [self.query(BQ_OFFSET, m) for m in range(self.count)] + [self.query(BQ_TOTAL_ROWS)]


def spmv_serve_create(batch_handle, n_streams, budget_bytes):
    h = ctypes.c_void_p()
    _check(lib.spmv_serve_create(batch_handle, int(n_streams), int(budget_bytes), ctypes.byref(h)))
    return h


def spmv_serve_destroy(h):
    _check(lib.spmv_serve_destroy(h))


def spmv_serve_run(h, matrix, width, seed, arrival_s, mode=SERVE_BATCHED, want_hash=True):
    """Run requests open loop; returns (latency_s, hashes or None, stats dict)."""
    m = np.ascontiguousarray(matrix, dtype=np.int32)
    w = np.ascontiguousarray(width, dtype=np.int32)
    sd = np.ascontiguousarray(seed, dtype=np.uint64)
    t = np.ascontiguousarray(arrival_s, dtype=np.float64)
    lat = np.zeros(m.size, dtype=np.float64)
    hs = np.zeros(m.size, dtype=np.uint64) if want_hash else None
    st = np.zeros(6, dtype=np.int64)
    _check(lib.spmv_serve_run(h, m.size, _ptr(m), _ptr(w), _ptr(sd), _ptr(t), int(mode), _ptr(lat),
                              _ptr(hs) if hs is not None else None, _ptr(st)))
    keys = ["blocks", "max_inflight", "waits_for_memory", "peak_pool_bytes", "elapsed_ns",
            "admitted_while_busy"]
    return lat, hs, dict(zip(keys, (int(v) for v in st)))


def spmv_serve_set_group_max(h, max_blocks):
    _check(lib.spmv_serve_set_group_max(h, int(max_blocks)))


def spmv_serve_pm1_bits(m):
    """Bits of m * 2^-52 - 1 (low 53 bits of m) as the request generator
    builds them; host only."""
    return int(lib.spmv_serve_pm1_bits(int(m) & 0xFFFFFFFFFFFFFFFF))


def spmv_serve_launches(h):
    out = ctypes.c_int64()
    _check(lib.spmv_serve_launches(h, ctypes.byref(out)))
    return out.value


def spmv_serve_single(h, matrix, width, seed, y_dev, x_dev, stream):
    _check(lib.spmv_serve_single(h, int(matrix), int(width), ctypes.c_uint64(int(seed)),
                                 _ptr(y_dev), _ptr(x_dev), _stream(stream)))


class Server:
    """Owns one serving runtime over a Batch of resident matrices."""

    def __init__(self, batch, n_streams=8, budget_bytes=40 << 30):
        self.batch = batch
        self.h = spmv_serve_create(batch.h, n_streams, budget_bytes)

    def close(self):
        if self.h is not None:
            spmv_serve_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, matrix, width, seed, arrival_s, mode=SERVE_BATCHED, want_hash=True):
        return spmv_serve_run(self.h, matrix, width, seed, arrival_s, mode, want_hash)
