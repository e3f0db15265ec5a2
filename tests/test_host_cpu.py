"""Host-side checks that need no GPU: the C ABI library builds, loads and
exports every function include/spmv.h declares, and the schedule enumerator
of the package agrees with the oracle's brute force (Sec. III-B/III-C)."""
import ctypes
import json
import os
import random

import numpy as np
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


def _header_params():
    """Parameter type lists of every function include/spmv.h declares."""
    import re
    from paper_2203_02530_gb300 import spmv
    text = re.sub(r"/\*.*?\*/", "", open(spmv.HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(?:int|int64_t|uint64_t|const char\*)\s+(spmv_\w+)\s*\(([^)]*)\)\s*;", text):
        params = [q.strip() for q in m.group(2).split(",") if q.strip() and q.strip() != "void"]
        out[m.group(1)] = [re.sub(r"\s*\b\w+$", "", q) if " " in q or "*" in q else q for q in params]
    return out


def test_binding_argtypes_match_the_header(libpath):
    """Every declared function is bound with as many arguments as the
    header gives it, each of the matching ctypes kind (64-bit integers,
    32-bit integers, pointers), so a binding cannot pass an argument in
    the wrong slot or width."""
    import ctypes as C
    from paper_2203_02530_gb300 import spmv
    decl = _header_params()
    assert set(decl) == set(spmv.declared_functions())
    for name, params in decl.items():
        argtypes = getattr(spmv.lib, name).argtypes or []
        assert len(argtypes) == len(params), (name, params, argtypes)
        for ctype, ptype in zip(argtypes, params):
            if "*" in ptype or ptype.endswith("_t stream") or ptype.startswith("cudaStream_t"):
                kind = "ptr"
            elif ptype.startswith(("int64_t", "uint64_t")):
                kind = "i64"
            elif ptype.startswith("int"):
                kind = "i32"
            else:
                kind = "other"
            want = {"ptr": (C.c_void_p,), "i64": (C.c_int64, C.c_uint64), "i32": (C.c_int,)}.get(kind)
            if want is None:
                continue
            ok = ctype in want or (kind == "ptr" and issubclass(ctype, (C._Pointer, C.c_void_p, C.c_char_p)))
            assert ok, (name, ptype, ctype)


def test_host_buffer_streams_reject_bad_arguments_without_a_gpu(libpath):
    """The streamed host-buffer entry points check their handle before any
    CUDA call."""
    from paper_2203_02530_gb300 import spmv
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_apply_host_many(None, 2, None, 0, None, 0, 0, None, None)
    assert e.value.code == spmv.EINVAL
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_batch_run_host_many(None, 2, None, 0, None, 0, 4, None, None, None)
    assert e.value.code == spmv.EINVAL


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
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_probe_dfma(10, 2, 32, None, 0, None)
    assert e.value.code == spmv.EINVAL
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_selftest_merge_abort(-5)
    assert e.value.code == spmv.EINVAL


@pytest.mark.parametrize("case,code", [
    ("n_negative", "EINVAL"), ("P_zero", "EINVAL"), ("P_over_limit", "EBOUNDS"), ("granularity", "EINVAL"),
    ("row_ptr_decreasing", "EINVAL"), ("column_out_of_range", "EINVAL"), ("column_negative", "EINVAL"),
    ("null_columns", "EINVAL"), ("n_over_int32", "EBOUNDS")])
def test_plan_rejects_malformed_input_without_a_gpu(libpath, case, code):
    """spmv_part_create checks the CSR and the partition count on the host,
    before any CUDA call, and returns the documented status."""
    from paper_2203_02530_gb300 import spmv
    n, P, gran = 4, 2, spmv.COARSE
    rp = np.array([0, 1, 2, 3, 4], np.int64)
    ci = np.array([0, 1, 2, 3], np.int32)
    va = np.ones(4)
    if case == "n_negative":
        n = -1
    elif case == "P_zero":
        P = 0
    elif case == "P_over_limit":
        P = 1025
    elif case == "granularity":
        gran = 7
    elif case == "row_ptr_decreasing":
        rp = np.array([0, 2, 1, 3, 4], np.int64)
    elif case == "column_out_of_range":
        ci = np.array([0, 1, 4, 3], np.int32)
    elif case == "column_negative":
        ci = np.array([0, -1, 2, 3], np.int32)
    elif case == "n_over_int32":
        n = 2**31
    if case == "null_columns":
        out = ctypes.c_void_p()
        st = spmv.lib.spmv_part_create(n, rp.ctypes.data_as(ctypes.c_void_p), None,
                                       va.ctypes.data_as(ctypes.c_void_p), P, gran, ctypes.byref(out))
        assert st == getattr(spmv, code) and not out.value
        return
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_part_create(n, rp, ci, va, P, gran)
    assert e.value.code == getattr(spmv, code), spmv.spmv_last_error()


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


def test_splitmix64_published_first_output():
    """SplitMix64 seeded with 0 first returns 0xE220A8397B1DCDAF (the
    generator of the serving requests' inputs)."""
    import numpy as np
    from paper_2203_02530_gb300 import workloads as W
    assert int(W.splitmix64(0, np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF
    x = W.request_x(99, 1000, 8)
    assert x.min() >= -1.0 and x.max() < 1.0 and abs(x.mean()) < 0.05


def test_request_draw_bits_equal_the_conversion(libpath):
    """The device generator builds 2u - 1 = m * 2^-52 - 1 from the bits of the
    53-bit draw m with integer operations; the host copy of that construction
    must equal converting m to double and subtracting 1, bit for bit, at the
    ends (m = 0 gives -1, m = 2^52 gives +0), at every exponent on both sides
    of zero, and on random draws."""
    import numpy as np
    from paper_2203_02530_gb300 import spmv
    ms = {0, 1, 2, 3, 2**52 - 1, 2**52, 2**52 + 1, 2**53 - 1}
    for b in range(53):
        for d in (-1, 0, 1):
            for m in (2**52 + (1 << b) + d, 2**52 - (1 << b) + d):
                if 0 <= m < 2**53:
                    ms.add(m)
    rng = np.random.default_rng(17)
    ms.update(int(v) for v in rng.integers(0, 2**53, size=2000, dtype=np.uint64))
    ms = np.array(sorted(ms), dtype=np.uint64)
    want = (ms.astype(np.float64) * 2.0 ** -53 * 2.0 - 1.0).view(np.uint64)
    got = np.array([spmv.spmv_serve_pm1_bits(int(m)) for m in ms], dtype=np.uint64)
    assert np.array_equal(got, want)
    assert spmv.spmv_serve_pm1_bits(2**52) == 0          # +0, not -0
    # only the low 53 bits are read
    assert spmv.spmv_serve_pm1_bits(2**63 + 5) == spmv.spmv_serve_pm1_bits(5)


def test_malformed_csr_rejected_before_any_cuda_call(libpath):
    """Host-side fault injection: bad plans are refused with SPMV_EINVAL /
    SPMV_EBOUNDS before the library touches the GPU."""
    import numpy as np
    from paper_2203_02530_gb300 import spmv
    bad = [(2, [0, 1, 2], [0, 5], [1.0, 1.0], 1, spmv.EINVAL),     # column out of range
           (2, [0, 2, 1], [0, 1], [1.0, 1.0], 1, spmv.EINVAL),     # decreasing row_ptr
           (2, [0, 1, 2], [0, 1], [1.0, 1.0], 0, spmv.EINVAL),     # P < 1
           (2, [0, 1, 2], [0, 1], [1.0, 1.0], 2000, spmv.EBOUNDS),  # P above the limit
           (-1, [0], [], [], 1, spmv.EINVAL)]
    for n, rp, ci, va, P, code in bad:
        with pytest.raises(spmv.SpmvError) as e:
            spmv.spmv_part_create(n, np.array(rp), np.array(ci, dtype=np.int32), np.array(va), P)
        assert e.value.code == code, (n, rp, P)
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_part_create(2, np.array([0, 1, 2]), np.array([0, 1], np.int32), np.ones(2), 1, 7)
    assert e.value.code == spmv.EINVAL


def test_record_log_resumes_without_remeasuring(tmp_path):
    """Checkpoint/resume of a search: measured programs are read back from
    the JSONL log and not measured again."""
    from paper_2203_02530_gb300 import search
    path = str(tmp_path / "log.jsonl")
    rec = search.Recorder(path, meta={"workload": "t"})
    rec.put([0, 1, 2, 3], [0, 0, 0, 0], 1.5e-4)
    rec.put([1, 0, 2, 3], [0, 1, 0, 1], 1.2e-4)
    again = search.Recorder(path)
    assert again.get([0, 1, 2, 3], [0, 0, 0, 0]) == 1.5e-4
    assert again.get((1, 0, 2, 3), (0, 1, 0, 1)) == 1.2e-4
    assert again.get([0, 2, 1, 3], [0, 0, 0, 0]) is None
    calls = []

    class FakePart:
        def run(self, *a, **k):
            calls.append(a)
            raise AssertionError("must not measure a recorded program")

    ev = search.graph_evaluator(FakePart(), [None], None, None, recorder=again)
    assert ev([0, 1, 2, 3], [0, 0, 0, 0]) == 1.5e-4
    assert not calls


def test_tuner_times_per_rank_plans_rank_by_rank(libpath, monkeypatch, tmp_path):
    """The variant tuner times a coarse plan's products as one launch over
    all ranks and a per-rank plan's as its P per-rank launches, skips the
    candidates a plan refuses (EINVAL), keeps the fastest, and keys its cache
    by granularity as well as by matrix and candidate set."""
    from paper_2203_02530_gb300 import autotune, spmv

    class FakePart:
        def __init__(self, P, gran):
            self.P, self.granularity, self.h = P, gran, object()
            self.set = []

        def set_op_variant(self, op, v, p):
            if v == spmv.VARIANT_MERGE:
                raise spmv.SpmvError(spmv.EINVAL, "refused")
            self.set.append((op, v, p))

    calls = []
    monkeypatch.setattr(spmv, "spmv_local", lambda h, p, x, y, s: calls.append(("L", p)))
    monkeypatch.setattr(spmv, "spmv_remote", lambda h, p, y, s: calls.append(("R", p)))
    cost = {(spmv.VARIANT_SELL, 8): 2.0, (spmv.VARIANT_SELL, 2008): 1.0, (spmv.VARIANT_PAIRS, 1): 3.0}
    current = {}

    def fake_time(run, stream, reps):
        before = len(calls)
        run()
        current["launches"] = calls[before:]
        return cost[current["vp"]]

    monkeypatch.setattr(autotune, "time_loop", fake_time)
    cands = [(spmv.VARIANT_SELL, 8), (spmv.VARIANT_MERGE, 0), (spmv.VARIANT_SELL, 2008), (spmv.VARIANT_PAIRS, 1)]
    orig_set = FakePart.set_op_variant

    def tracking_set(self, op, v, p):
        orig_set(self, op, v, p)
        current["vp"] = (v, p)

    monkeypatch.setattr(FakePart, "set_op_variant", tracking_set)
    cache = str(tmp_path / "tune.json")
    for gran, ranks in ((spmv.COARSE, [-1]), (spmv.PER_PARTITION, [0, 1, 2])):
        part = FakePart(3, gran)
        calls.clear()
        r = autotune.tune(part, None, None, None, sig="sig", candidates=cands, cache_path=cache)
        assert r["local"] == (spmv.VARIANT_SELL, 2008) and r["remote"] == (spmv.VARIANT_SELL, 2008)
        assert all((op, spmv.VARIANT_MERGE, 0) not in r["times"] for op in (spmv.OP_LOCAL, spmv.OP_REMOTE))
        assert [p for k, p in current["launches"]] == ranks
        assert {k for k, p in calls} == {"L", "R"}
    keys = list(json.load(open(cache)).keys())
    assert len(keys) == 2 and sum("per-rank" in k for k in keys) == 1


def test_enumerator_matches_brute_force_on_random_dags():
    """Property check: on random DAGs of up to 6 operations and 1-3 streams
    the package's enumerator yields exactly the oracle's brute-force set of
    canonical schedules (all orders x all stream maps, filtered for
    topological order and canonical stream numbering), and counts it."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    @settings(max_examples=60, deadline=None, derandomize=True)
    @given(m=st.integers(1, 6), streams=st.integers(1, 3), bits=st.integers(0, 2**15 - 1))
    def prop(m, streams, bits):
        pairs = [(u, v) for u in range(m) for v in range(u + 1, m)]
        edges = [e for k, e in enumerate(pairs) if bits >> k & 1]
        ops = list(range(m))
        want = set(S.brute_force_schedules(ops, edges, streams))
        dag = E.Dag(m, edges)
        got = {(tuple(o), tuple(s)) for o, s in E.enumerate_schedules(dag, streams)}
        assert got == want
        assert E.count_schedules(dag, streams) == len(want)

    prop()
