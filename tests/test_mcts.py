"""Monte-Carlo tree search (Sec. III-C) on small DAGs, with synthetic
program times: it measures every implementation exactly once before it
stops, visits exactly the enumerator's (and the oracle's brute-force) set,
and keeps the exploitation value within [0, 1] (Sec. III-C.1)."""
import hashlib
import math

import pytest

from oracle import schedules as OS
from paper_2203_02530_gb300 import mcts as M
from paper_2203_02530_gb300 import schedules as E


def fake_time(order, smap):
    """Deterministic pseudo-time of a program (stands in for a measurement)."""
    key = ("%s|%s" % (order, smap)).encode()
    return 1.0 + int(hashlib.sha256(key).hexdigest()[:8], 16) / 2.0 ** 32


def run_to_end(dag, streams, seed):
    seen = []
    tree = M.Mcts(dag, streams, lambda o, s: (seen.append((tuple(o), tuple(s))), fake_time(o, s))[1],
                  seed=seed)
    vs = []
    it = 0
    while tree.iterate() is not None:
        it += 1
        if it in (3, 10, 30, 100):
            vs.extend(tree.exploit_values())
    vs.extend(tree.exploit_values())
    return tree, seen, vs


@pytest.mark.parametrize("streams", [1, 2, 3])
def test_coarse_dag_every_program_once(streams):
    ops, edges = OS.coarse_dag()
    dag = E.Dag(4, edges)
    tree, seen, vs = run_to_end(dag, streams, seed=streams)
    want = set(OS.brute_force_schedules(ops, edges, streams))
    assert len(seen) == len(set(seen)) == len(want)
    assert set(seen) == want
    assert tree.finished and tree.iterate() is None
    assert all(0.0 <= v <= 1.0 for v in vs)


def test_per_partition_dag_every_program_once():
    # per-rank DAG with P = 2 on one stream: 630 programs
    ops, edges = OS.per_partition_dag(2, lambda q, p: True)
    dag = E.Dag(len(ops), edges)
    tree, seen, vs = run_to_end(dag, 1, seed=7)
    assert len(seen) == len(set(seen)) == E.count_schedules(dag, 1) == 630
    assert set(seen) == {(tuple(o), tuple(s)) for o, s in E.enumerate_schedules(dag, 1)}
    assert all(0.0 <= v <= 1.0 for v in vs)


def test_budgeted_search_records_distinct_valid_programs():
    ops, edges = OS.per_partition_dag(3, lambda q, p: (p + q) % 2 == 1)
    dag = E.Dag(len(ops), edges)
    tree = M.Mcts(dag, 4, fake_time, seed=3)
    recs = tree.run(300)
    assert len(recs) == 300
    keys = {(tuple(o), tuple(s)) for o, s, _ in recs}
    assert len(keys) == 300
    for o, s, t in recs:
        assert dag.is_topological(o)
        assert OS.is_canonical_streams(o, s, set(ops))
        assert t == fake_time(o, s)
    # the root saw every rollout and the extreme times
    assert tree.root.n == 300
    assert tree.root.tmin == min(t for _, _, t in recs)
    assert tree.root.tmax == max(t for _, _, t in recs)


def test_exploit_value_definition():
    class N:
        pass
    parent, child = N(), N()
    parent.n, parent.tmin, parent.tmax = 5, 1.0, 3.0
    child.n, child.tmin, child.tmax = 2, 1.5, 2.5
    assert M.exploit_value(child, parent) == pytest.approx(0.5)
    child.n = 1
    assert M.exploit_value(child, parent) == 1.0
    child.n, parent.n = 2, 1
    assert M.exploit_value(child, parent) == 1.0
    assert M.C_EXPLORE == pytest.approx(math.sqrt(2))


def test_selection_prefers_wide_subtrees():
    """With equal visit counts the child whose times span more of the
    parent's range scores higher."""
    ops, edges = OS.coarse_dag()
    dag = E.Dag(4, edges)
    tree = M.Mcts(dag, 2, fake_time, seed=0)
    root = tree.root
    a = tree._child(root, root.legal[0])
    b = tree._child(root, root.legal[1])
    root.n, root.tmin, root.tmax = 8, 1.0, 2.0
    a.n, a.tmin, a.tmax = 4, 1.0, 1.9
    b.n, b.tmin, b.tmax = 4, 1.4, 1.5
    assert tree._score(a, root) > tree._score(b, root)
    b.explored = True
    assert tree._score(b, root) == -math.inf
