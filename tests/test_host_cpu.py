"""Host-side checks that need no GPU: the C ABI library builds, loads and
exports every function include/spmv.h declares, and the schedule enumerator
of the package agrees with the oracle's brute force (Sec. III-B/III-C)."""
import ctypes
import os
import random

import pytest

from oracle import schedules as S
from paper_2203_02530_gb300 import build as B
from paper_2203_02530_gb300 import schedules as E


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_library_exports_every_declared_function(libpath):
    from paper_2203_02530_gb300 import spmv
    lib = ctypes.CDLL(libpath)
    names = spmv.declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wires up exactly the declared functions
    for n in names:
        assert callable(getattr(spmv, n)), n


def test_last_error_is_empty_string_initially(libpath):
    from paper_2203_02530_gb300 import spmv
    assert isinstance(spmv.spmv_last_error(), str)


def test_invalid_arguments_fail_without_a_gpu(libpath):
    """Host-side argument checks run before any CUDA call."""
    from paper_2203_02530_gb300 import spmv
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_part_query(None, spmv.Q_N)
    assert e.value.code == spmv.EINVAL
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_csr_merge(-1, 0, 0, 0, 0, 0, 0, None)
    assert e.value.code == spmv.EINVAL
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_csr_merge(2**30, 2**30, 0, 0, 0, 0, 0, None)
    assert e.value.code == spmv.EBOUNDS


@pytest.mark.parametrize("streams", [1, 2, 3, 4])
def test_enumerator_matches_brute_force_coarse(streams):
    ops, edges = S.coarse_dag()
    want = set(S.brute_force_schedules(ops, edges, streams))
    dag = E.Dag(4, edges)
    got = {(tuple(o), tuple(s)) for o, s in E.enumerate_schedules(dag, streams)}
    assert got == want
    assert E.count_schedules(dag, streams) == len(want)


@pytest.mark.parametrize("P,streams", [(2, 1), (2, 2)])
def test_enumerator_matches_brute_force_per_partition(P, streams):
    sends = lambda q, p: (q + p) % 3 != 0
    ops, edges = S.per_partition_dag(P, sends)
    want = S.count_brute_force(ops, edges, streams)
    dag = E.Dag(len(ops), edges)
    assert E.count_schedules(dag, streams) == want
    got = list(E.enumerate_schedules(dag, streams))
    assert len(got) == want
    for o, s in random.Random(0).sample(got, min(50, len(got))):
        assert S.is_topological(o, edges)
        assert S.is_canonical_streams(o, s, set(ops))


def test_enumerator_small_dags():
    for ops, edges in [([0, 1, 2], []), ([0, 1, 2, 3], [(0, 1), (0, 2), (1, 3), (2, 3)]),
                       ([0, 1, 2, 3, 4], [(0, 4), (1, 4), (2, 3)])]:
        for st in (1, 2, 3):
            want = set(S.brute_force_schedules(ops, edges, st))
            dag = E.Dag(len(ops), edges)
            got = {(tuple(o), tuple(s)) for o, s in E.enumerate_schedules(dag, st)}
            assert got == want


def test_canonicalize():
    # op 2 comes first and its stream becomes 0; op 0 then opens stream 1
    assert E.canonicalize([2, 0, 1, 3], [1, 1, 0, 3]) == [1, 1, 0, 2]
