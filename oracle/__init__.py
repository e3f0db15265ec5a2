"""CPU oracle for the row-partitioned SpMV of Pearson, Javeed and Devine,
"Machine Learning for CUDA+MPI Design Rules" (Sec. III-A, Fig. 3).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it; the only thing both sides use is
the seeded input generator module, which holds none of the method's
arithmetic.

Contents:
  * ``OraclePlan`` / ``csr_spmv`` / ``csr_absdot``: ctypes bindings of the
    plain C implementation in ``spmv_oracle.c`` (the definition y = A x, the
    partition A = A_L + A_R of Sec. III-A, the pack / exchange / local /
    remote operations of Fig. 3c).
  * ``schedules``: the schedule space of Sec. III-B/III-C (topological
    traversals, stream binding with bijection pruning, Table III
    synchronisation) by brute force over permutations.
  * ``mcts_ref``: none; the search is host driver code in the package and is
    checked against ``schedules``' brute force.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None

# array selectors of orc_plan_export (mirrors the enum in spmv_oracle.c)
BOUNDS, L_PTR, L_COL, L_VAL, R_PTR, R_COL, R_VAL, HALO, SEND_IDX, HALO_OFF, \
    SEG_OFF, SENDBUF, RECVBUF = range(13)
_DTYPES = {BOUNDS: np.int64, L_PTR: np.int64, L_COL: np.int32,
           L_VAL: np.float64, R_PTR: np.int64, R_COL: np.int32,
           R_VAL: np.float64, HALO: np.int32, SEND_IDX: np.int32,
           HALO_OFF: np.int64, SEG_OFF: np.int64, SENDBUF: np.float64,
           RECVBUF: np.float64}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.orc_csr_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_csr_absdot.argtypes = [i64, vp, vp, vp, vp, vp]
        L.orc_csr_spmv_rows_parallel.argtypes = [i64, vp, vp, vp, vp, vp, i32]
        L.orc_max_threads.argtypes = []
        L.orc_plan_create.argtypes = [i64, vp, vp, vp, i32, ctypes.POINTER(vp)]
        L.orc_plan_destroy.argtypes = [vp]
        L.orc_plan_destroy.restype = None
        L.orc_plan_len.argtypes = [vp, i32, i32]
        L.orc_plan_len.restype = i64
        L.orc_plan_export.argtypes = [vp, i32, i32, vp, i64]
        L.orc_pack.argtypes = [vp, i32, vp]
        L.orc_copy.argtypes = [vp, i32]
        L.orc_local.argtypes = [vp, i32, vp, vp]
        L.orc_remote.argtypes = [vp, i32, vp]
        L.orc_partitioned_spmv.argtypes = [vp, vp, vp]
        L.orc_clear_buffers.argtypes = [vp]
        L.orc_clear_buffers.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col_idx, vals):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64),
            np.ascontiguousarray(col_idx, dtype=np.int32),
            np.ascontiguousarray(vals, dtype=np.float64))


def csr_spmv(n, row_ptr, col_idx, vals, x):
    """y = A x by the definition, rows in order (Sec. III-A, Fig. 3a)."""
    rp, ci, va = _csr(row_ptr, col_idx, vals)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    rc = lib().orc_csr_spmv(n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    if rc:
        raise ValueError("orc_csr_spmv failed: %d" % rc)
    return y


def csr_spmv_rows_parallel(n, row_ptr, col_idx, vals, x, threads=0):
    """csr_spmv with the rows shared among host threads (same result bit for
    bit); for timing the oracle on every core."""
    rp, ci, va = _csr(row_ptr, col_idx, vals)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    rc = lib().orc_csr_spmv_rows_parallel(n, _p(rp), _p(ci), _p(va), _p(x), _p(y), int(threads))
    if rc:
        raise ValueError("orc_csr_spmv_rows_parallel failed: %d" % rc)
    return y


def max_threads():
    """Threads the parallel product uses by default (1 without OpenMP)."""
    return int(lib().orc_max_threads())


def csr_absdot(n, row_ptr, col_idx, vals, x):
    """sum_j |a_ij x_j| per row: the scale of the dot-product error bound."""
    rp, ci, va = _csr(row_ptr, col_idx, vals)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(n, dtype=np.float64)
    rc = lib().orc_csr_absdot(n, _p(rp), _p(ci), _p(va), _p(x), _p(out))
    if rc:
        raise ValueError("orc_csr_absdot failed: %d" % rc)
    return out


class OraclePlan:
    """The partition plan of Fig. 3b and the four per-rank operations.

    ``P`` ranks own rows floor(p n / P) .. floor((p+1) n / P).  Operations
    take ``part`` = a rank, or -1 for every rank at once (the coarse op).
    """

    def __init__(self, n, row_ptr, col_idx, vals, P):
        self.n, self.P = int(n), int(P)
        self._keep = _csr(row_ptr, col_idx, vals)
        h = ctypes.c_void_p()
        rc = lib().orc_plan_create(self.n, *(_p(a) for a in self._keep),
                                   self.P, ctypes.byref(h))
        if rc:
            raise ValueError("orc_plan_create failed: %d" % rc)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_plan_destroy(self._h)
            self._h = None

    __del__ = close

    def export(self, what, p=-1):
        n = lib().orc_plan_len(self._h, what, p)
        if n < 0:
            raise ValueError("bad export selector")
        out = np.empty(n, dtype=_DTYPES[what])
        rc = lib().orc_plan_export(self._h, what, p, _p(out), n)
        if rc:
            raise ValueError("export failed")
        return out

    def bounds(self):
        return self.export(BOUNDS)

    def halo(self, p):
        return self.export(HALO, p)

    def pack(self, q, x):
        self._x = np.ascontiguousarray(x, dtype=np.float64)
        _check(lib().orc_pack(self._h, q, _p(self._x)))

    def copy(self, p):
        _check(lib().orc_copy(self._h, p))

    def local(self, p, x, y):
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert y.dtype == np.float64 and y.flags.c_contiguous
        _check(lib().orc_local(self._h, p, _p(x), _p(y)))

    def remote(self, p, y):
        assert y.dtype == np.float64 and y.flags.c_contiguous
        _check(lib().orc_remote(self._h, p, _p(y)))

    def clear_buffers(self):
        lib().orc_clear_buffers(self._h)

    def spmv(self, x):
        """y = A_L x_L + A_R x_R in the order pack, local, copy, remote."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n, dtype=np.float64)
        _check(lib().orc_partitioned_spmv(self._h, _p(x), _p(y)))
        return y

    def run_op(self, kind, part, x, y):
        """Run one DAG operation (kind in pack/local/copy/remote)."""
        if kind == "pack":
            self.pack(part, x)
        elif kind == "local":
            self.local(part, x, y)
        elif kind == "copy":
            self.copy(part)
        elif kind == "remote":
            self.remote(part, y)
        else:
            raise ValueError(kind)


def _check(rc):
    if rc:
        raise ValueError("oracle call failed: %d" % rc)
