"""Implementations of an operation DAG: topological orders with a stream
binding per operation (Sec. III-B, Eq. 1; Table II BoundGPU vertices),
pruned of stream relabellings (Sec. III-C.2).

Canonical form: streams are numbered by first use along the order, so the
first operation is on stream 0 and every operation uses a stream already in
use or the next unused number.  The enumerator walks prefixes P_k depth
first (the sequential-decision view of Sec. III-B), extending a prefix by
every ready operation on every admissible stream.
"""
import math
from functools import lru_cache


class Dag:
    """Operations 0..n_ops-1 and dependency edges (u, v): u before v."""

    def __init__(self, n_ops, edges):
        self.n_ops = int(n_ops)
        self.edges = [(int(u), int(v)) for u, v in edges]
        self.pred_mask = [0] * self.n_ops
        for u, v in self.edges:
            self.pred_mask[v] |= 1 << u

    def ready(self, done_mask):
        """Operations not yet issued whose predecessors all are."""
        return [v for v in range(self.n_ops)
                if not done_mask >> v & 1 and self.pred_mask[v] & done_mask == self.pred_mask[v]]

    def is_topological(self, order):
        done = 0
        if sorted(order) != list(range(self.n_ops)):
            return False
        for v in order:
            if self.pred_mask[v] & done != self.pred_mask[v]:
                return False
            done |= 1 << v
        return True


def coarse_spmv_dag():
    """pack -> copy -> remote, local -> remote (op ids 0..3 = pack, local,
    copy, remote)."""
    return Dag(4, [(0, 2), (2, 3), (1, 3)])


def children(dag, done_mask, n_used, n_streams):
    """Legal next decisions (op, stream) from a prefix: every ready op on a
    stream already used or the next unused one."""
    out = []
    for v in dag.ready(done_mask):
        for s in range(min(n_used + 1, n_streams)):
            out.append((v, s))
    return out


def enumerate_schedules(dag, n_streams, limit=None):
    """Yield (order, stream_of_op) for every canonical implementation."""
    order, smap = [], [0] * dag.n_ops
    count = [0]

    def rec(done, n_used):
        if limit is not None and count[0] >= limit:
            return
        if len(order) == dag.n_ops:
            count[0] += 1
            yield list(order), list(smap)
            return
        for v, s in children(dag, done, n_used, n_streams):
            order.append(v)
            smap[v] = s
            yield from rec(done | 1 << v, max(n_used, s + 1))
            order.pop()

    yield from rec(0, 0)


def count_schedules(dag, n_streams):
    """Number of canonical implementations, by dynamic programming over
    (issued set, streams in use)."""

    @lru_cache(maxsize=None)
    def f(done, n_used):
        if done == (1 << dag.n_ops) - 1:
            return 1
        return sum(f(done | 1 << v, max(n_used, s + 1))
                   for v, s in children(dag, done, n_used, n_streams))

    return f(0, 0)


def canonicalize(order, stream_of_op):
    """Relabel streams by first use along the order."""
    remap, out = {}, list(stream_of_op)
    for v in order:
        s = stream_of_op[v]
        if s not in remap:
            remap[s] = len(remap)
        out[v] = remap[s]
    return out


def stirling2(m, k):
    return sum((-1) ** j * math.comb(k, j) * (k - j) ** m for j in range(k + 1)) // math.factorial(k)
