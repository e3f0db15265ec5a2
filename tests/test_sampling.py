"""Random sampling of implementations, the search baseline of Sec. VI
(uniform random sampling set against MCTS at an equal number of measured
programs).  The uniform sampler is checked against the oracle's brute-force
set and the enumerator's count, and its draws against the uniform
distribution by a chi-squared test at a fixed seed; the per-decision
sampler (random legal decisions, the rollout of Sec. III-C without a
tree) is shown to be a different distribution."""
import collections
import random

import pytest

from oracle import schedules as OS
from paper_2203_02530_gb300 import schedules as E


def _dag(ops_edges):
    ops, edges = ops_edges
    return E.Dag(len(ops), edges)


def _chi2_crit(df, p=1e-4):
    stats = pytest.importorskip("scipy.stats")
    return float(stats.chi2.ppf(1.0 - p, df))


def _chi2(counts, keys, draws):
    exp = draws / len(keys)
    return sum((counts.get(k, 0) - exp) ** 2 / exp for k in keys)


@pytest.mark.parametrize("case,streams", [("coarse", 1), ("coarse", 2), ("coarse", 3),
                                          ("pp2", 1)])
def test_total_equals_brute_force(case, streams):
    oe = OS.coarse_dag() if case == "coarse" else OS.per_partition_dag(2, lambda q, p: True)
    want = OS.count_brute_force(oe[0], oe[1], streams)
    assert E.UniformSampler(_dag(oe), streams).total() == want


@pytest.mark.parametrize("P,streams", [(2, 2), (3, 2), (3, 3)])
def test_total_equals_subset_dp(P, streams):
    dag = _dag(OS.per_partition_dag(P, lambda q, p: (q + p) % 3 != 0))
    assert E.UniformSampler(dag, streams).total() == E.count_schedules(dag, streams)


def test_stream_map_counts_closed_forms():
    # one stream: one binding; unlimited streams (S >= r): the Bell numbers;
    # S = 2: 2^(r-1) bindings of r operations from none in use
    g = E.stream_map_counts(6, 6)
    assert [g[r][0] for r in range(7)] == [1, 1, 2, 5, 15, 52, 203]
    assert all(E.stream_map_counts(r, 1)[r][0] == 1 for r in range(6))
    assert all(E.stream_map_counts(r, 2)[r][0] == 2 ** (r - 1) for r in range(1, 8))


@pytest.mark.parametrize("case,streams,per_prog", [("coarse", 2, 600), ("pp2", 1, 60)])
def test_uniform_sampler_is_uniform(case, streams, per_prog):
    oe = OS.coarse_dag() if case == "coarse" else OS.per_partition_dag(2, lambda q, p: True)
    dag = _dag(oe)
    keys = set(OS.brute_force_schedules(oe[0], oe[1], streams))
    sampler = E.UniformSampler(dag, streams)
    rng = random.Random(12345)
    draws = per_prog * len(keys)
    counts = collections.Counter()
    for _ in range(draws):
        o, m = sampler.draw(rng)
        k = (tuple(o), tuple(m))
        assert k in keys          # valid: topological and canonical
        counts[k] += 1
    assert set(counts) == keys    # every program drawn
    assert _chi2(counts, keys, draws) < _chi2_crit(len(keys) - 1)


def test_per_decision_sampler_is_not_uniform():
    """On the coarse DAG the first decision is PACK or LOCAL with equal
    probability per decision, but only 1 of the 3 orders starts with LOCAL."""
    dag = _dag(OS.coarse_dag())
    rng = random.Random(7)
    n = 6000
    per_dec = sum(E.draw_per_decision(dag, 1, rng)[0][0] == OS.LOCAL for _ in range(n)) / n
    sampler = E.UniformSampler(dag, 1)
    uni = sum(sampler.draw(rng)[0][0] == OS.LOCAL for _ in range(n)) / n
    assert abs(per_dec - 0.5) < 0.03
    assert abs(uni - 1.0 / 3.0) < 0.03


@pytest.mark.parametrize("mode", ["uniform", "per_decision"])
def test_sample_programs_distinct_valid_and_exact_count(mode):
    oe = OS.per_partition_dag(2, lambda q, p: True)
    dag = _dag(oe)
    keys = set(OS.brute_force_schedules(oe[0], oe[1], 1))
    got = E.sample_programs(dag, 1, 200, seed=3, mode=mode)
    assert len(got) == 200
    ks = [(tuple(o), tuple(m)) for o, m in got]
    assert len(set(ks)) == 200 and set(ks) <= keys
    everything = E.sample_programs(dag, 1, 10_000, seed=3, mode=mode)   # more than exist
    assert set((tuple(o), tuple(m)) for o, m in everything) == keys and len(everything) == len(keys)


def test_random_sampling_measures_each_program_once():
    from paper_2203_02530_gb300 import search   # loads the library
    class FakePart:
        n_ops = 8
        def dag(self):
            return OS.per_partition_dag(2, lambda q, p: True)[1]
    calls = []

    def evaluate(o, m):
        calls.append((tuple(o), tuple(m)))
        return 1.0 + len(calls) * 1e-3

    recs = search.random_sampling(FakePart(), [0, 1], evaluate, 50, seed=9)
    assert len(recs) == 50 and len(set(calls)) == 50 and len(calls) == 50
    assert [r[2] for r in recs] == [1.0 + (i + 1) * 1e-3 for i in range(50)]


def test_uniform_sampler_on_the_power_law_dag():
    """The per-rank DAG of 8 ranks that all send to each other (32 ops):
    the order count is checked against a closed form for its structure on
    two ranks, and draws are valid programs."""
    dag = _dag(OS.per_partition_dag(8, lambda q, p: True))
    sampler = E.UniformSampler(dag, 4)
    rng = random.Random(1)
    for _ in range(20):
        o, m = sampler.draw(rng)
        assert OS.is_topological(o, dag.edges)
        assert OS.is_canonical_streams(o, m, set(range(32)))
        assert max(m) < 4
    assert sampler.total() == sampler.orders() * E.stream_map_counts(32, 4)[32][0]
