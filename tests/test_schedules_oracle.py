"""Pins of the oracle's schedule space (Sec. III-B/III-C, Table III):
closed forms, the paper's two printed traversals, Table III itself, and the
invariance of y over every valid order (oracle run on the CPU)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import schedules as S
from paper_2203_02530_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def stirling2(m, k):
    return sum((-1) ** j * math.comb(k, j) * (k - j) ** m for j in range(k + 1)) // math.factorial(k)


def partitions_le(m, s):
    return sum(stirling2(m, k) for k in range(0, s + 1)) if m else 1


@pytest.mark.parametrize("streams,count", [(1, 3), (2, 24), (4, 45)])
def test_coarse_dag_closed_form(streams, count):
    """3 topological orders (local anywhere before remote) times the set
    partitions of 4 ops into at most S streams."""
    ops, edges = S.coarse_dag()
    assert S.count_brute_force(ops, edges, streams) == count
    assert count == 3 * partitions_le(4, streams)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_antichain_single_stream_is_factorial(m):
    assert S.count_brute_force(list(range(m)), [], 1) == math.factorial(m)


@pytest.mark.parametrize("m,s", [(3, 2), (4, 3), (5, 2), (4, 4)])
def test_chain_counts_set_partitions(m, s):
    ops = list(range(m))
    edges = [(i, i + 1) for i in range(m - 1)]
    assert S.count_brute_force(ops, edges, s) == partitions_le(m, s)


def test_diamond():
    # 0 -> {1, 2} -> 3: two orders, times partitions of 4 ops into <= 2
    ops, edges = [0, 1, 2, 3], [(0, 1), (0, 2), (1, 3), (2, 3)]
    assert S.count_brute_force(ops, edges, 2) == 2 * 8


def test_canonical_form_prunes_exactly_the_bijections():
    """Each canonical schedule stands for S!/(S-k)! labelled ones, k = the
    streams it uses: summing gives every labelled map of valid orders."""
    ops, edges = S.coarse_dag()
    for s in (2, 3):
        canon = S.brute_force_schedules(ops, edges, s)
        total = 0
        for order, smap in canon:
            k = len(set(smap))
            total += math.perm(s, k)
        orders = [o for o in itertools.permutations(ops) if S.is_topological(o, edges)]
        assert total == len(orders) * s ** 4


def test_paper_printed_traversals_are_valid():
    g = json.load(open(os.path.join(GOLD, "paper_traversals.json")))
    v, edges, kind = S.paper_fig3c_dag()
    for t in g["traversals"]:
        assert S.is_topological(t, edges)
    a, b = g["edge_needing_sync"]["edge"]
    assert (a, b) in edges
    assert kind[a] == "GPU" and kind[b] == "CPU"
    assert S.sync_for_edge(kind[a], 0, kind[b], None) != []
    # swapping Pack after PostSends, or y_R before WaitRecv, is invalid
    t = list(g["traversals"][0])
    t[1], t[3] = t[3], t[1]
    assert not S.is_topological(t, edges)
    t = list(g["traversals"][1])
    i7, i8 = t.index(7), t.index(8)
    t[i7], t[i8] = t[i8], t[i7]
    assert not S.is_topological(t, edges)


def test_table3():
    g = json.load(open(os.path.join(GOLD, "table3_sync.json")))
    for row in g["rows"]:
        if row["same_stream"] is None:
            us, vs = (0 if row["u"] == "GPU" else None), (1 if row["v"] == "GPU" else None)
        else:
            us, vs = 0, (0 if row["same_stream"] else 1)
        assert S.sync_for_edge(row["u"], us, row["v"], vs) == row["inserted"]


def test_sync_names_follow_paper_convention():
    v, edges, kind = S.paper_fig3c_dag()
    names = {1: "start", 2: "Pack", 3: "yL", 4: "PostSend", 5: "PostRecv",
             6: "WaitSend", 7: "WaitRecv", 8: "yR", 9: "combine", 10: "end"}
    smap = {k: (0 if kind[k] == "GPU" else None) for k in v}
    seq = S.sync_op_names([1, 2, 3, 4, 5, 6, 7, 8, 9, 10], smap, edges, names, kind)
    assert "CER-after-Pack" in seq and "CES-b4-PostSend" in seq
    assert seq.index("CER-after-Pack") < seq.index("CES-b4-PostSend") < seq.index("PostSend")


def test_sync_counts_coarse():
    ops, edges = S.coarse_dag()
    # pack, copy on stream 0; local, remote on stream 1: edges pack->copy
    # same stream; copy->remote and local->remote: only copy->remote crosses
    rec, waits, syncs = S.sync_counts(edges, [0, 1, 0, 1])
    assert (rec, waits, syncs) == (1, 1, 0)
    rec, waits, syncs = S.sync_counts(edges, [0, 0, 0, 0])
    assert (rec, waits, syncs) == (0, 0, 0)
    rec, waits, syncs = S.sync_counts(edges, [0, 1, 2, 3])
    assert (rec, waits, syncs) == (3, 3, 0)


def _random_topo(ops, edges, rng):
    pred = {v: set() for v in ops}
    for u, v in edges:
        pred[v].add(u)
    done, order = set(), []
    while len(order) < len(ops):
        ready = sorted(v for v in ops if v not in done and pred[v] <= done)
        v = ready[rng.integers(len(ready))]
        order.append(v)
        done.add(v)
    return order


def test_every_valid_order_gives_the_same_y_on_the_oracle():
    """Schedule invariance: any topological order of the per-rank DAG run
    on the oracle's CPU operations gives bit-identical y; an order that
    breaks the copy -> remote edge does not."""
    n, rp, ci, va = W.powerlaw(2000, seed=8, cap=100)
    x = W.uniform_x(n, seed=9)
    P = 4
    pl = oracle.OraclePlan(n, rp, ci, va, P)
    seg = pl.export(oracle.SEG_OFF)
    ops, edges = S.per_partition_dag(P, lambda q, p: seg[p * P + q + 1] > seg[p * P + q])
    ref = pl.spmv(x)
    rng = np.random.default_rng(0)
    for _ in range(30):
        order = _random_topo(ops, edges, rng)
        assert S.is_topological(order, edges)
        pl.clear_buffers()
        y = np.full(n, np.nan)
        for op in order:
            pl.run_op(S.KIND_NAMES[op % 4], op // 4, x, y)
        assert np.array_equal(y, ref)
    # remote of rank 1 before its copy: reads a cleared receive buffer
    order = _random_topo(ops, edges, rng)
    i_copy, i_rem = order.index(4 * 1 + S.COPY), order.index(4 * 1 + S.REMOTE)
    order[i_copy], order[i_rem] = order[i_rem], order[i_copy]
    assert not S.is_topological(order, edges)
    pl.clear_buffers()
    y = np.full(n, np.nan)
    for op in order:
        pl.run_op(S.KIND_NAMES[op % 4], op // 4, x, y)
    assert not np.array_equal(y, ref)


def test_per_partition_dag_small_count():
    """Per-rank DAG with P = 2, 1 stream: the number of topological orders
    equals a direct count of linear extensions."""
    ops, edges = S.per_partition_dag(2, lambda q, p: True)
    n1 = S.count_brute_force(ops, edges, 1)
    # independent count: dynamic programming over subsets
    pred = {v: 0 for v in ops}
    for u, v in edges:
        pred[v] |= 1 << u
    f = {0: 1}
    for mask in range(1 << len(ops)):
        if mask not in f:
            continue
        for v in ops:
            if not mask >> v & 1 and pred[v] & mask == pred[v]:
                f[mask | 1 << v] = f.get(mask | 1 << v, 0) + f[mask]
    assert n1 == f[(1 << len(ops)) - 1]


def test_per_segment_dag_structure():
    """One PACK and one COPY per (destination, source) segment: each PACK
    feeds only its COPY, each COPY only its destination's REMOTE, and every
    REMOTE also waits for its rank's LOCAL."""
    P = 3
    sends = lambda q, p: (q, p) != (0, 2)   # every ordered pair but 0 -> 2
    ops, edges, segs = S.per_segment_dag(P, sends)
    assert segs == [(p, q) for p in range(P) for q in range(P) if q != p and sends(q, p)]
    assert len(ops) == 2 * P + 2 * len(segs)
    E = set(edges)
    assert len(E) == len(edges) == P + 2 * len(segs)
    for p in range(P):
        assert (2 * p, 2 * p + 1) in E
    for k, (p, q) in enumerate(segs):
        pack, copy = 2 * P + 2 * k, 2 * P + 2 * k + 1
        assert (pack, copy) in E and (copy, 2 * p + 1) in E
        assert [e for e in edges if e[0] == pack] == [(pack, copy)]
        assert [e for e in edges if e[0] == copy] == [(copy, 2 * p + 1)]


def test_per_segment_dag_small_count():
    """P = 2, both directions, one stream: the library's enumerator, a brute
    force over all permutations and a subset DP agree on the number of
    topological orders of the 8-op DAG."""
    from paper_2203_02530_gb300 import schedules as E
    ops, edges, segs = S.per_segment_dag(2, lambda q, p: True)
    assert len(ops) == 8 and len(segs) == 2
    n1 = S.count_brute_force(ops, edges, 1)
    pred = {v: 0 for v in ops}
    for u, v in edges:
        pred[v] |= 1 << u
    f = {0: 1}
    for mask in range(1 << len(ops)):
        if mask not in f:
            continue
        for v in ops:
            if not mask >> v & 1 and pred[v] & mask == pred[v]:
                f[mask | 1 << v] = f.get(mask | 1 << v, 0) + f[mask]
    assert n1 == f[(1 << len(ops)) - 1]
    assert E.count_schedules(E.Dag(len(ops), edges), 1) == n1
