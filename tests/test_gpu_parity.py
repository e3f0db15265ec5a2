"""GPU parity: every kernel, operation and schedule of the library against
the CPU oracle, through the C ABI.

Plan arrays, pack and exchange buffers are compared bit for bit; y within
the FP64 dot-product bound 1e-12 * sum_j |a_ij x_j| (exactly for integer
data); every valid schedule must give a bit-identical y."""
import random

import numpy as np
import pytest

import oracle
from oracle import schedules as OS
from paper_2203_02530_gb300 import workloads as W
from tests.gpu_util import assert_fp64_close, dev, reference, refill, synced, torch_cuda

pytestmark = pytest.mark.gpu


def _dense_row_matrix():
    # one row holding 20000 entries among short rows: longer than a tile
    # stage and spread over many merge tiles
    n = 20000
    rng = np.random.default_rng(21)
    lens = rng.integers(0, 6, size=n)
    lens[777] = n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    cols = []
    for i in range(n):
        c = np.arange(n) if lens[i] == n else np.sort(rng.choice(n, size=lens[i], replace=False))
        cols.append(c)
    ci = np.concatenate(cols).astype(np.int32)
    va = rng.uniform(-1, 1, size=ci.size)
    return n, rp, ci, va


def _empty_rows():
    n = 1000
    rp = np.zeros(n + 1, dtype=np.int64)
    return n, rp, np.zeros(0, np.int32), np.zeros(0)


CASES = {
    "lap64": (lambda: W.laplacian_5pt(64), 2),
    "st27_20": (lambda: W.stencil_27pt(20, seed=1), 4),
    "st27_ragged": (lambda: W.stencil_27pt(0, seed=3, dims=(7, 13, 29)), 3),
    "powerlaw": (lambda: W.powerlaw(40000, seed=3), 8),
    "rand_dup": (lambda: W.random_csr(300, density=0.05, seed=4, duplicates=True,
                                      shuffle_cols=True), 3),
    "dense_row": (_dense_row_matrix, 4),
    "empty_rows": (_empty_rows, 2),
    "tiny_P_gt_n": (lambda: W.random_csr(5, density=0.6, seed=5), 8),
    "one": (lambda: W.random_csr(1, density=1.0, seed=6, empty_rows=False), 1),
    "band": (lambda: W.band(15000, 150000, 3750, seed=7), 4),
}
_cache = {}


def case(name):
    if name not in _cache:
        gen, P = CASES[name]
        n, rp, ci, va = gen()
        x = W.uniform_x(n, seed=99)
        _cache[name] = (n, rp, ci, va, P, x)
    return _cache[name]


VARIANTS = ([("tile", g) for g in range(5)] + [("vector", v) for v in (2, 4, 8, 16, 32)]
            + [("pairs", v) for v in (1, 2, 4, 8, 102, 104)] + [("warp", g) for g in range(5)]
            + [("merge", 0)] + [("sell", u) for u in (4, 8, 9, 104, 105, 106, 107, 2004, 2009, 2104, 2106)])

SELL_LONG = 64


def _sell_rank(lens):
    """Padded entries of one rank's rows in the sliced layout: rows longer
    than SELL_LONG are summed elsewhere; natural order unless padding each
    32-row slice to its longest short row adds more than 1/8 (+1024), then
    the short rows sorted by length."""
    short = lens <= SELL_LONG
    nat = 0
    for s0 in range(0, lens.size, 32):
        blk = lens[s0:s0 + 32][short[s0:s0 + 32]]
        nat += 32 * int(blk.max()) if blk.size else 0
    sn = int(lens[short].sum())
    if nat <= sn + sn // 8 + 1024:
        return nat
    srt = np.sort(lens[short])[::-1]
    return sum(32 * int(srt[s0]) for s0 in range(0, srt.size, 32))


def sell_entries(part, P):
    """Padded entries of the sliced layout, from the exported plan: each
    rank's local rows and its rows with remote entries."""
    from paper_2203_02530_gb300 import spmv
    tot = 0
    for p in range(P):
        ll = np.diff(part.export(spmv.X_L_PTR, p))
        rl = np.diff(part.export(spmv.X_R_PTR, p))
        tot += _sell_rank(ll) + _sell_rank(rl[rl > 0])
    return tot


def make_part(n, rp, ci, va, P, gran=0):
    from paper_2203_02530_gb300 import spmv
    return spmv.Part(n, rp, ci, va, P, gran)


def set_variant(part, v):
    from paper_2203_02530_gb300 import spmv
    kind, param = v
    code = {"tile": spmv.VARIANT_TILE, "vector": spmv.VARIANT_VECTOR,
            "merge": spmv.VARIANT_MERGE, "pairs": spmv.VARIANT_PAIRS,
            "warp": spmv.VARIANT_WARP, "sell": spmv.VARIANT_SELL}[kind]
    part.set_variant(code, param)
    if kind == "sell":
        assert part.query(spmv.Q_SELL_ENTRIES) == sell_entries(part, part.query(spmv.Q_P))


def run_default(part, x_d, y_d, stream):
    """pack, local, copy, remote on one stream (the default schedule)."""
    from paper_2203_02530_gb300 import spmv
    spmv.spmv_pack(part.h, -1, x_d, stream)
    spmv.spmv_local(part.h, -1, x_d, y_d, stream)
    spmv.spmv_halo_copy(part.h, -1, stream)
    spmv.spmv_remote(part.h, -1, y_d, stream)


# ------------------------------------------------------------------ plan
@pytest.mark.parametrize("name", sorted(CASES))
def test_plan_arrays_bit_exact(name):
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    n, rp, ci, va, P, x = case(name)
    ref = oracle.OraclePlan(n, rp, ci, va, P)
    with make_part(n, rp, ci, va, P) as part:
        pairs = [(spmv.X_BOUNDS, oracle.BOUNDS), (spmv.X_SEND_IDX, oracle.SEND_IDX),
                 (spmv.X_HALO_OFF, oracle.HALO_OFF), (spmv.X_SEG_OFF, oracle.SEG_OFF)]
        for a, b in pairs:
            assert np.array_equal(part.export(a), ref.export(b)), a
        per = [(spmv.X_L_PTR, oracle.L_PTR), (spmv.X_L_COL, oracle.L_COL),
               (spmv.X_L_VAL, oracle.L_VAL), (spmv.X_R_PTR, oracle.R_PTR),
               (spmv.X_R_COL, oracle.R_COL), (spmv.X_R_VAL, oracle.R_VAL),
               (spmv.X_HALO, oracle.HALO)]
        for p in range(P):
            for a, b in per:
                assert np.array_equal(part.export(a, p), ref.export(b, p)), (a, p)
        assert part.query(spmv.Q_NNZ) == rp[-1] - rp[0]
        assert part.query(spmv.Q_NNZ_LOCAL) + part.query(spmv.Q_NNZ_REMOTE) == rp[-1] - rp[0]


# ------------------------------------------------------------------ pack / copy
@pytest.mark.parametrize("name", ["lap64", "st27_ragged", "powerlaw", "rand_dup", "tiny_P_gt_n"])
def test_pack_and_copy_bit_exact(name):
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    ref = oracle.OraclePlan(n, rp, ci, va, P)
    s = torch.cuda.Stream()
    x_d = dev(x)
    with make_part(n, rp, ci, va, P) as part:
        # coarse
        spmv.spmv_pack(part.h, -1, x_d, s)
        spmv.spmv_halo_copy(part.h, -1, s)
        s.synchronize()
        ref.pack(-1, x)
        ref.copy(-1)
        assert np.array_equal(part.export(spmv.X_SENDBUF), ref.export(oracle.SENDBUF))
        assert np.array_equal(part.export(spmv.X_RECVBUF), ref.export(oracle.RECVBUF))
        # per rank, in an interleaved order, on a fresh vector
        x2 = W.uniform_x(n, seed=5)
        x2_d = dev(x2)
        ref.clear_buffers()
        for q in reversed(range(P)):
            spmv.spmv_pack(part.h, q, x2_d, s)
            ref.pack(q, x2)
        for p in range(P):
            spmv.spmv_halo_copy(part.h, p, s)
            ref.copy(p)
        s.synchronize()
        assert np.array_equal(part.export(spmv.X_SENDBUF), ref.export(oracle.SENDBUF))
        assert np.array_equal(part.export(spmv.X_RECVBUF), ref.export(oracle.RECVBUF))


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: "%s%d" % v)
@pytest.mark.parametrize("name", sorted(CASES))
def test_product_parity_every_variant(name, variant):
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    y_d = synced(torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device="cuda"))
    with make_part(n, rp, ci, va, P) as part:
        set_variant(part, variant)
        run_default(part, x_d, y_d, s)
        s.synchronize()
        y1 = y_d.cpu().numpy()[:n].copy()
        assert_fp64_close(y1, want, scale, "%s %s" % (name, variant))
        run_default(part, x_d, y_d, s)
        s.synchronize()
        assert np.array_equal(y_d.cpu().numpy()[:n], y1), "not deterministic"
        assert part.query(spmv.Q_ERROR) == 0


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: "%s%d" % v)
def test_integer_data_is_exact(variant):
    torch = torch_cuda()
    n, rp, ci, va = W.random_csr(2500, density=0.004, seed=8, integer=True, duplicates=True)
    x = W.uniform_x(n, seed=9, integer=True)
    want = oracle.csr_spmv(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, 5) as part:
        set_variant(part, variant)
        run_default(part, x_d, y_d, s)
        s.synchronize()
        assert np.array_equal(y_d.cpu().numpy(), want)


@pytest.mark.parametrize("name", ["lap64", "st27_20", "st27_ragged", "band", "rand_dup"])
def test_sliced_layout_matches_thread_per_row_bit_for_bit(name):
    """SELL and WARP both sum each row from 0.0 in storage order with one FMA
    per entry, so their y agree bit for bit (padding adds nothing)."""
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    s = torch.cuda.Stream()
    x_d = dev(x)
    out = []
    for v in (("warp", 0), ("sell", 4), ("sell", 9), ("sell", 104), ("sell", 2008), ("sell", 2104)):
        y_d = synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))
        with make_part(n, rp, ci, va, P) as part:
            set_variant(part, v)
            run_default(part, x_d, y_d, s)
            s.synchronize()
        out.append(y_d.cpu().numpy())
    for o in out[1:]:
        assert np.array_equal(out[0].view(np.uint64), o.view(np.uint64))


@pytest.mark.parametrize("name", sorted(CASES))
def test_sell16_local_matches_sell_bit_for_bit(name):
    """16-bit column deltas change only the index bytes: the LOCAL product
    gives SELL's y bit for bit (and the oracle's within the bound)."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    out = []
    with make_part(n, rp, ci, va, P) as part:
        part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_SELL, 4)
        for v in (spmv.VARIANT_SELL, spmv.VARIANT_SELL16):
            part.set_op_variant(spmv.OP_LOCAL, v, 9)
            assert part.query(spmv.Q_LOCAL_VARIANT) == 100 * v + 9
            y_d = synced(torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device="cuda"))
            run_default(part, x_d, y_d, s)
            s.synchronize()
            out.append(y_d.cpu().numpy()[:n])
        assert part.query(spmv.Q_ERROR) == 0
        with pytest.raises(spmv.SpmvError):
            part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_SELL16, 4)
        with pytest.raises(spmv.SpmvError):
            part.set_variant(spmv.VARIANT_SELL16, 4)
    assert np.array_equal(out[0].view(np.uint64), out[1].view(np.uint64))
    assert_fp64_close(out[1], want, scale, "%s sell16" % name)


def test_sell16_refused_when_a_delta_needs_more_than_16_bits():
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    n = 70000
    rp = np.arange(n + 1, dtype=np.int64)
    ci = ((np.arange(n) + 40000) % n).astype(np.int32)   # every column 40000 rows away (mod n)
    va = np.ones(n)
    with make_part(n, rp, ci, va, 1) as part:
        with pytest.raises(spmv.SpmvError) as e:
            part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL16, 9)
        assert e.value.code == spmv.EINVAL
        assert part.query(spmv.Q_LOCAL_VARIANT) // 100 != spmv.VARIANT_SELL16


def _lengths_matrix(lens, seed):
    """Rows of the given lengths with distinct random columns."""
    rng = np.random.default_rng(seed)
    n = len(lens)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    ci = np.concatenate([np.sort(rng.choice(n, size=k, replace=False)) for k in lens]).astype(np.int32) \
        if rp[-1] else np.zeros(0, np.int32)
    return n, rp, ci, rng.uniform(-1, 1, size=ci.size)


@pytest.mark.parametrize("lens_kind", ["all_long", "edge_64_65", "long_and_empty", "one_long_in_natural",
                                       "cut_rows"])
@pytest.mark.parametrize("gran", [0, 1])
@pytest.mark.parametrize("param", [4, 2104])
def test_sliced_layout_edge_cases(lens_kind, gran, param):
    """Rows at and around the 64-entry long-row threshold, ranks made of long
    rows only, empty rows among long ones, a single long row inside a
    natural-order rank (a hole in its slice), and rows cut into 512-entry
    pieces, coarse and per rank, with round-robin and cost-balanced CTA
    ranges; twice, so the pieces' counters are reset."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    rng = np.random.default_rng(31)
    n = 700
    if lens_kind == "all_long":
        lens = rng.integers(65, 300, size=n)
    elif lens_kind == "edge_64_65":
        lens = rng.choice([63, 64, 65, 66], size=n)
    elif lens_kind == "long_and_empty":
        lens = np.where(rng.random(n) < 0.5, 0, rng.integers(65, 200, size=n))
    elif lens_kind == "one_long_in_natural":
        lens = np.full(n, 9)
        lens[333] = 500
    else:   # rows cut into 512-entry pieces, including exact multiples
        lens = rng.integers(1, 20, size=3000)
        lens[::37] = rng.choice([513, 1024, 1025, 2999], size=lens[::37].size)
    n, rp, ci, va = _lengths_matrix(lens, 32)
    x = W.uniform_x(n, seed=33)
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    y_d = synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))
    P = 3
    with make_part(n, rp, ci, va, P, gran) as part:
        set_variant(part, ("sell", param))
        if gran == 0:
            run_default(part, x_d, y_d, s)
        else:
            for p in range(P):
                spmv.spmv_pack(part.h, p, x_d, s)
            for p in range(P):
                spmv.spmv_local(part.h, p, x_d, y_d, s)
                spmv.spmv_halo_copy(part.h, p, s)
            for p in reversed(range(P)):
                spmv.spmv_remote(part.h, p, y_d, s)
        s.synchronize()
        y1 = y_d.cpu().numpy().copy()
        assert_fp64_close(y1, want, scale, "sliced %s gran %d" % (lens_kind, gran))
        refill(y_d)
        run_default(part, x_d, y_d, s)
        s.synchronize()
        assert np.array_equal(y_d.cpu().numpy(), y1)
        assert part.query(spmv.Q_ERROR) == 0


@pytest.mark.parametrize("name", ["st27_ragged", "powerlaw", "dense_row"])
def test_local_and_remote_variants_chosen_separately(name):
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, P) as part:
        for lv, rv in [((spmv.VARIANT_PAIRS, 2), (spmv.VARIANT_MERGE, 0)),
                       ((spmv.VARIANT_MERGE, 0), (spmv.VARIANT_VECTOR, 8)),
                       ((spmv.VARIANT_TILE, 4), (spmv.VARIANT_PAIRS, 4))]:
            part.set_op_variant(spmv.OP_LOCAL, *lv)
            part.set_op_variant(spmv.OP_REMOTE, *rv)
            assert part.query(spmv.Q_LOCAL_VARIANT) == 100 * lv[0] + lv[1]
            assert part.query(spmv.Q_REMOTE_VARIANT) == 100 * rv[0] + rv[1]
            refill(y_d)
            run_default(part, x_d, y_d, s)
            s.synchronize()
            assert_fp64_close(y_d.cpu().numpy(), want, scale, "%s %s %s" % (name, lv, rv))
        with pytest.raises(spmv.SpmvError):
            part.set_op_variant(spmv.OP_PACK, spmv.VARIANT_TILE, 0)


# ------------------------------------------------------------------ schedules
def _sync_expect(dag_edges, smap):
    rec, waits, _ = OS.sync_counts(dag_edges, smap)
    return rec, waits


@pytest.mark.parametrize("name", ["lap64", "st27_20", "powerlaw"])
def test_every_coarse_schedule_gives_identical_y(name):
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(2)]
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, P) as part:
        edges = part.dag()
        assert sorted(edges) == sorted(OS.coarse_dag()[1])
        scheds = list(E.enumerate_schedules(E.Dag(4, edges), 2))
        assert len(scheds) == 24
        first = None
        for order, smap in scheds:
            refill(y_d)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)
            assert (part.query(spmv.Q_LAST_RECORDS), part.query(spmv.Q_LAST_WAITS)) == \
                _sync_expect(edges, smap)
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
            torch.cuda.synchronize()
            ye = y_d.cpu().numpy().copy()
            refill(y_d)
            torch.cuda.synchronize()
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            torch.cuda.synchronize()
            yg = y_d.cpu().numpy()
            assert np.array_equal(ye, yg)
            if first is None:
                first = ye
                assert_fp64_close(ye, want, scale, name)
            assert np.array_equal(ye, first), (order, smap)
            spmv.spmv_graph_destroy(part.h, g)


def _random_schedule(dag, n_streams, rng):
    done, used, order, smap = 0, 0, [], [0] * dag.n_ops
    while len(order) < dag.n_ops:
        ready = dag.ready(done)
        v = ready[rng.randrange(len(ready))]
        s = rng.randrange(min(used + 1, n_streams))
        order.append(v)
        smap[v] = s
        used = max(used, s + 1)
        done |= 1 << v
    return order, smap


@pytest.mark.parametrize("name,variant", [("st27_ragged", ("sell", 9)), ("powerlaw", ("sell", 4)),
                                          ("band", ("vector", 2)), ("tiny_P_gt_n", ("tile", 0)),
                                          ("lap64", ("pairs", 2))])
def test_per_segment_granularity(name, variant):
    """One PACK and one COPY per halo segment: the DAG is the oracle's
    per-segment reading, op ids decode as documented, every random schedule
    (eager and captured) gives the same y bit for bit, and the send and
    receive buffers equal the oracle's."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    ref = oracle.OraclePlan(n, rp, ci, va, P)
    seg = ref.export(oracle.SEG_OFF)
    ops, oedges, segs = OS.per_segment_dag(P, lambda q, p: seg[p * P + q + 1] > seg[p * P + q])
    streams = [torch.cuda.Stream() for _ in range(3)]
    x_d = dev(x)
    y_d = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, P, spmv.PER_SEGMENT) as part:
        set_variant(part, variant)
        assert part.n_ops == len(ops)
        assert sorted(map(tuple, part.dag())) == sorted(oedges)
        for op in ops:
            kind, d, sr = spmv.spmv_part_op_info(part.h, op)
            if op < 2 * P:
                assert (kind, d, sr) == ((spmv.OP_LOCAL, spmv.OP_REMOTE)[op % 2], op // 2, -1)
            else:
                p_, q_ = segs[(op - 2 * P) // 2]
                assert (kind, d, sr) == ((spmv.OP_PACK, spmv.OP_COPY)[op % 2], p_, q_)
        ref.pack(-1, x)
        ref.copy(-1)
        dag = E.Dag(len(ops), oedges)
        rng = random.Random(5)
        first = None
        for trial in range(6):
            order, smap = _random_schedule(dag, 3, rng)
            refill(y_d)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)
            torch.cuda.synchronize()
            ye = y_d.cpu().numpy()[:n].copy()
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
            refill(y_d)
            torch.cuda.synchronize()
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            torch.cuda.synchronize()
            assert np.array_equal(y_d.cpu().numpy()[:n], ye)
            spmv.spmv_graph_destroy(part.h, g)
            if first is None:
                first = ye
                assert_fp64_close(ye, want, scale, "%s per segment" % name)
                assert np.array_equal(part.export(spmv.X_SENDBUF), ref.export(oracle.SENDBUF))
                assert np.array_equal(part.export(spmv.X_RECVBUF), ref.export(oracle.RECVBUF))
            assert np.array_equal(ye, first), (order, smap)
        assert part.query(spmv.Q_ERROR) == 0


@pytest.mark.parametrize("name,variant", [("st27_ragged", ("tile", 0)), ("powerlaw", ("merge", 0)),
                                          ("powerlaw", ("tile", 2)), ("band", ("vector", 4)),
                                          ("powerlaw", ("sell", 4)), ("dense_row", ("sell", 9)),
                                          ("powerlaw", ("sell", 2104)), ("dense_row", ("sell", 2008))])
def test_per_partition_schedules_give_identical_y(name, variant):
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    ref = oracle.OraclePlan(n, rp, ci, va, P)
    seg = ref.export(oracle.SEG_OFF)
    streams = [torch.cuda.Stream() for _ in range(4)]
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, P, spmv.PER_PARTITION) as part:
        set_variant(part, variant)
        edges = part.dag()
        _, oedges = OS.per_partition_dag(P, lambda q, p: seg[p * P + q + 1] > seg[p * P + q])
        assert sorted(edges) == sorted(oedges)
        dag = E.Dag(4 * P, edges)
        rng = random.Random(1)
        first = None
        for it in range(24):
            order, smap = _random_schedule(dag, 4, rng)
            refill(y_d)
            if it % 2:
                g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
                part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            else:
                part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)
                assert (part.query(spmv.Q_LAST_RECORDS), part.query(spmv.Q_LAST_WAITS)) == \
                    _sync_expect(edges, smap)
            torch.cuda.synchronize()
            y = y_d.cpu().numpy().copy()
            if it % 2:
                spmv.spmv_graph_destroy(part.h, g)
            if first is None:
                first = y
                assert_fp64_close(y, want, scale, name)
            assert np.array_equal(y, first), (order, smap)


@pytest.mark.parametrize("name,gran,variant", [
    ("powerlaw", 1, ("sell", 2009)), ("powerlaw", 1, ("merge", 0)), ("st27_ragged", 1, ("vector", 4)),
    ("st27_20", 0, ("sell", 107)), ("rand_dup", 2, ("tile", 0)), ("powerlaw", 2, ("sell", 104))])
def test_relaxed_mode_gives_identical_y(name, gran, variant):
    """SPMV_RUN_RELAXED lets the ops without DAG predecessors overlap the
    kernel before them on their stream: random schedules on 1 to 4 streams,
    captured, every replay into a NaN-filled y, give y bit-identical to the
    default (stream-ordered) mode, eager and captured, and within the
    oracle's bound; the relaxed flag is refused for eager issue."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(4)]
    x_d = dev(x)
    y_d = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, P, gran) as part:
        set_variant(part, variant)
        dag = E.Dag(part.n_ops, part.dag())
        rng = random.Random(5)
        first = None
        for it in range(12):
            order, smap = _random_schedule(dag, 1 + it % 4, rng)
            for flags in (spmv.RUN_EAGER, spmv.RUN_CAPTURE, spmv.RUN_CAPTURE | spmv.RUN_RELAXED):
                g = None
                reps = 3 if flags & spmv.RUN_CAPTURE else 1
                if flags & spmv.RUN_CAPTURE:
                    g = part.run(order, smap, streams, x_d, y_d, flags)
                for _ in range(reps):
                    refill(y_d)
                    if g is None:
                        part.run(order, smap, streams, x_d, y_d, flags)
                    else:
                        part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
                    torch.cuda.synchronize()
                    y = y_d.cpu().numpy()[:n].copy()
                    if first is None:
                        first = y
                        assert_fp64_close(y, want, scale, name)
                    assert np.array_equal(y.view(np.uint64), first.view(np.uint64)), (order, smap, flags)
                if g is not None:
                    spmv.spmv_graph_destroy(part.h, g)
        with pytest.raises(spmv.SpmvError) as e:
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER | spmv.RUN_RELAXED)
        assert e.value.code == spmv.EINVAL
        assert part.query(spmv.Q_ERROR) == 0


def _local_then_remote_program(part):
    """Packs and copies on stream 1, then each rank's local and remote
    products in turn on stream 0: every remote product follows its rank's
    local product on its stream (the case SPMV_RUN_DEFER overlaps)."""
    from paper_2203_02530_gb300 import spmv
    info = [spmv.spmv_part_op_info(part.h, v) for v in range(part.n_ops)]
    order = ([v for v in range(part.n_ops) if info[v][0] == spmv.OP_PACK]
             + [v for v in range(part.n_ops) if info[v][0] == spmv.OP_COPY])
    smap = [1] * part.n_ops
    for d in sorted({i[1] for i in info if i[0] == spmv.OP_LOCAL}):
        for kind in (spmv.OP_LOCAL, spmv.OP_REMOTE):
            v = [u for u in range(part.n_ops) if info[u][0] == kind and info[u][1] == d][0]
            order.append(v)
            smap[v] = 0
    return order, smap


@pytest.mark.parametrize("name,gran,local,remote", [
    ("st27_20", 0, ("sell", 107), ("sell", 107)), ("st27_20", 0, ("sell16", 9), ("sell", 8)),
    ("powerlaw", 1, ("sell", 2009), ("sell", 2104)), ("powerlaw", 1, ("merge", 0), ("sell", 8)),
    ("powerlaw", 2, ("sell", 104), ("sell", 104)), ("st27_ragged", 1, ("vector", 4), ("sell", 4)),
    ("rand_dup", 1, ("sell", 8), ("sell", 9)), ("empty_rows", 1, ("sell", 4), ("sell", 4)),
    ("st27_20", 1, ("sell", 9), ("pairs", 2))])
def test_defer_mode_gives_identical_y(name, gran, local, remote):
    """SPMV_RUN_DEFER lets a sliced remote product read A_R and the halo and
    sum its rows before waiting for the kernel before it on its stream (when
    that kernel writes none of its inputs but y): random programs on 1 to 4
    streams and the program that puts each rank's remote product right after
    its local product, captured and replayed into NaN-filled y, give y
    bit-identical to the stream-ordered mode and within the oracle's bound;
    that program defers every non-empty remote product (none when the remote
    variant is not sliced); the same with SPMV_RUN_RELAXED as well; the flag
    is refused for eager issue."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(4)]
    x_d = dev(x)
    y_d = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    code = {"sell": spmv.VARIANT_SELL, "sell16": spmv.VARIANT_SELL16, "merge": spmv.VARIANT_MERGE,
            "vector": spmv.VARIANT_VECTOR, "pairs": spmv.VARIANT_PAIRS}
    sliced = remote[0] == "sell"
    with make_part(n, rp, ci, va, P, gran) as part:
        part.set_op_variant(spmv.OP_LOCAL, code[local[0]], local[1])
        part.set_op_variant(spmv.OP_REMOTE, code[remote[0]], remote[1])
        dag = E.Dag(part.n_ops, part.dag())
        rng = random.Random(9)
        first = None

        def check(order, smap, flags, reps):
            nonlocal first
            g = part.run(order, smap, streams, x_d, y_d, flags) if flags & spmv.RUN_CAPTURE else None
            deferred = part.query(spmv.Q_LAST_DEFERRED)
            for _ in range(reps):
                refill(y_d)
                if g is None:
                    part.run(order, smap, streams, x_d, y_d, flags)
                else:
                    part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
                torch.cuda.synchronize()
                y = y_d.cpu().numpy()[:n].copy()
                if first is None:
                    first = y
                    assert_fp64_close(y, want, scale, name)
                assert np.array_equal(y.view(np.uint64), first.view(np.uint64)), (order, smap, flags)
            if g is not None:
                spmv.spmv_graph_destroy(part.h, g)
            return deferred

        order, smap = _local_then_remote_program(part)
        check(order, smap, spmv.RUN_EAGER, 1)
        deferred = check(order, smap, spmv.RUN_CAPTURE | spmv.RUN_DEFER, 5)
        assert check(order, smap, spmv.RUN_CAPTURE | spmv.RUN_DEFER | spmv.RUN_RELAXED, 5) == deferred
        remote_ops = sum(1 for v in range(part.n_ops)
                         if spmv.spmv_part_op_info(part.h, v)[0] == spmv.OP_REMOTE)
        if not sliced:
            assert deferred == 0
        elif name != "empty_rows":
            assert deferred == remote_ops, (deferred, remote_ops)
        total = 0
        for it in range(12):
            order, smap = _random_schedule(dag, 1 + it % 4, rng)
            check(order, smap, spmv.RUN_CAPTURE, 1)
            total += check(order, smap, spmv.RUN_CAPTURE | spmv.RUN_DEFER, 3)
            check(order, smap, spmv.RUN_CAPTURE | spmv.RUN_DEFER | spmv.RUN_RELAXED, 2)
        if not sliced:
            assert total == 0
        for bad in (spmv.RUN_EAGER | spmv.RUN_DEFER, spmv.RUN_EAGER | spmv.RUN_RELAXED | spmv.RUN_DEFER):
            with pytest.raises(spmv.SpmvError) as e:
                part.run(order, smap, streams, x_d, y_d, bad)
            assert e.value.code == spmv.EINVAL
        assert part.query(spmv.Q_ERROR) == 0


@pytest.mark.parametrize("name,gran", [("lap64", 0), ("st27_20", 1), ("st27_ragged", 0), ("powerlaw", 1),
                                       ("powerlaw", 0), ("rand_dup", 1)])
def test_release_csr_keeps_y_and_restores(name, gran):
    """spmv_part_release_csr frees the CSR copy once both products are
    sliced (the long rows move to compact arrays): less device memory, y
    bit-identical eager and captured; exporting the matrix arrays rebuilds
    the CSR bit for bit; the index check passes; a CSR variant afterwards
    still gives the oracle's y; and the call is refused while a product is
    not sliced or while graphs exist."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    mats = (spmv.X_L_COL, spmv.X_L_VAL, spmv.X_R_COL, spmv.X_R_VAL)
    with make_part(n, rp, ci, va, P, gran) as part:
        order = [op for k in (0, 1, 2, 3) for op in range(part.n_ops)
                 if spmv.spmv_part_op_info(part.h, op)[0] == k]
        smap = [0] * part.n_ops

        def product(flags=spmv.RUN_EAGER):
            refill(y_d)
            if flags == spmv.RUN_EAGER:
                part.run(order, smap, [s], x_d, y_d)
            else:
                g = part.run(order, smap, [s], x_d, y_d, flags)
                part.run(order, smap, [s], x_d, y_d, spmv.RUN_REPLAY, g)
                s.synchronize()
                spmv.spmv_graph_destroy(part.h, g)
            torch.cuda.synchronize()
            return y_d.cpu().numpy().copy()

        part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_SELL, 8)
        with pytest.raises(spmv.SpmvError) as e:   # LOCAL not sliced yet
            part.release_csr()
        assert e.value.code == spmv.EINVAL
        try:
            part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL16, 9)
        except spmv.SpmvError:
            part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL, 9)
        y0 = product()
        assert_fp64_close(y0, want, scale, name)
        before = {(w, p): part.export(w, p) for w in mats for p in range(P)}
        bytes0 = part.query(spmv.Q_DEVICE_BYTES)
        part.release_csr()
        bytes1 = part.query(spmv.Q_DEVICE_BYTES)
        # 12 bytes per entry freed, less the compact copy of the long rows
        assert bytes0 - bytes1 >= 4 * part.query(spmv.Q_NNZ)
        for flags in (spmv.RUN_EAGER, spmv.RUN_CAPTURE, spmv.RUN_CAPTURE | spmv.RUN_RELAXED):
            assert np.array_equal(product(flags).view(np.uint64), y0.view(np.uint64)), flags
        after = {(w, p): part.export(w, p) for w in mats for p in range(P)}   # rebuilds the CSR
        for k in before:
            assert before[k].dtype == after[k].dtype and np.array_equal(
                before[k].view(np.uint8), after[k].view(np.uint8)), k
        assert part.query(spmv.Q_DEVICE_BYTES) >= bytes0 - 1024
        assert spmv.spmv_part_check(part.h) == 0
        assert np.array_equal(product().view(np.uint64), y0.view(np.uint64))
        part.release_csr()
        g = part.run(order, smap, [s], x_d, y_d, spmv.RUN_CAPTURE)
        with pytest.raises(spmv.SpmvError) as e:   # graphs hold the arrays
            part.release_csr()
        spmv.spmv_graph_destroy(part.h, g)
        part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_VECTOR, 4)   # needs the CSR: rebuilt
        assert_fp64_close(product(), want, scale, name + " after restore")
        assert part.query(spmv.Q_ERROR) == 0


def test_invalid_schedules_are_rejected_before_launch():
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case("lap64")
    streams = [torch.cuda.Stream() for _ in range(2)]
    x_d = dev(x)
    y_d = synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))
    with make_part(n, rp, ci, va, P) as part:
        bad = [([2, 0, 1, 3], [0, 0, 0, 0]),    # copy before pack
               ([0, 2, 3, 1], [0, 0, 0, 0]),    # remote before local
               ([0, 1, 2, 3], [0, 2, 0, 0]),    # stream out of range
               ([0, 1, 2, 2], [0, 0, 0, 0]),    # op repeated
               ([0, 1, 2], [0, 0, 0])]          # op missing
        for order, smap in bad:
            with pytest.raises(spmv.SpmvError) as e:
                part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)
            assert e.value.code == spmv.ESCHED
        torch.cuda.synchronize()
        assert np.isnan(y_d.cpu().numpy()).all(), "something ran"
        with pytest.raises(spmv.SpmvError) as e:
            spmv.spmv_pack(part.h, P, x_d, streams[0])
        assert e.value.code == spmv.EINVAL


# ------------------------------------------------------------------ standalone merge
@pytest.mark.parametrize("name", sorted(CASES))
def test_standalone_merge_product(name):
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    if rp[0] != 0:
        pytest.skip("needs row_ptr[0] == 0")
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    # exact-size tensors: the kernel must stay inside each array
    rp_d = dev(rp.astype(np.int32))
    ci_d = dev(ci) if ci.size else torch.empty(0, dtype=torch.int32, device="cuda")
    va_d = dev(va) if va.size else torch.empty(0, dtype=torch.float64, device="cuda")
    x_d = dev(x) if n else torch.empty(0, dtype=torch.float64, device="cuda")
    y_d = synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))
    spmv.spmv_csr_merge(n, int(rp[-1]), rp_d, ci_d, va_d, x_d, y_d, s)
    s.synchronize()
    assert_fp64_close(y_d.cpu().numpy(), want, scale, name)
    y1 = y_d.cpu().numpy().copy()
    spmv.spmv_csr_merge(n, int(rp[-1]), rp_d, ci_d, va_d, x_d, y_d, s)
    s.synchronize()
    assert np.array_equal(y_d.cpu().numpy(), y1)
    assert spmv.spmv_csr_error() == 0


def test_standalone_merge_rejects_misaligned():
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case("lap64")
    rp_d = dev(rp.astype(np.int32))
    big = synced(torch.zeros(ci.size + 1, dtype=torch.int32, device="cuda"))
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_csr_merge(n, int(rp[-1]), rp_d, big[1:], dev(va), dev(x),
                            torch.empty(n, dtype=torch.float64, device="cuda"), None)
    assert e.value.code == spmv.EINVAL


# ------------------------------------------------------------------ host buffers
def test_apply_host_buffers():
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case("st27_20")
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    with make_part(n, rp, ci, va, P) as part:
        xi, yi = spmv.spmv_part_io_buffers(part.h)
        g = part.run([0, 1, 2, 3], [0, 0, 0, 0], [s], xi, yi, spmv.RUN_CAPTURE)
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty(n, dtype=torch.float64).pin_memory()
        spmv.spmv_apply_host(part.h, g, xh, yh, s)
        assert_fp64_close(yh.numpy(), want, scale, "host path")
        with pytest.raises(spmv.SpmvError):
            g2 = part.run([0, 1, 2, 3], [0, 0, 0, 0], [s], dev(x), yi, spmv.RUN_CAPTURE)
            spmv.spmv_apply_host(part.h, g2, xh, yh, s)


@pytest.mark.parametrize("name,variant", [("st27_ragged", ("sell", 9)), ("powerlaw", ("sell", 4)),
                                          ("tiny_P_gt_n", ("vector", 2)), ("empty_rows", ("tile", 0))])
def test_apply_host_pipelined_matches_graph_path(name, variant):
    """Block-wise x transfers overlapped with the LOCAL products give the
    graph path's y bit for bit."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    want, scale = reference(n, rp, ci, va, x)
    s, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with make_part(n, rp, ci, va, P) as part:
        set_variant(part, variant)
        xi, yi = spmv.spmv_part_io_buffers(part.h)
        g = part.run([0, 1, 2, 3], [0, 0, 0, 0], [s], xi, yi, spmv.RUN_CAPTURE)
        xh = torch.from_numpy(x).pin_memory()
        y1 = torch.full((max(n, 1),), float("nan"), dtype=torch.float64).pin_memory()
        y2 = torch.full((max(n, 1),), float("nan"), dtype=torch.float64).pin_memory()
        spmv.spmv_apply_host(part.h, g, xh, y1, s)
        spmv.spmv_apply_host_pipelined(part.h, xh, y2, s, s2)
        a, b = y1.numpy()[:n], y2.numpy()[:n]
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
        assert_fp64_close(b, want, scale, "pipelined host path")
        with pytest.raises(spmv.SpmvError):
            spmv.spmv_apply_host_pipelined(part.h, xh, y2, s, s)


@pytest.mark.parametrize("name,variant", [("st27_ragged", ("sell", 9)), ("powerlaw", ("sell", 4)),
                                          ("tiny_P_gt_n", ("vector", 2)), ("empty_rows", ("tile", 0))])
def test_apply_host_many_matches_single_products(name, variant):
    """A stream of independent products through host buffers, consecutive
    ones overlapped on two pairs of device vectors: every y_k equals the
    single pipelined product of x_k bit for bit, whether the host vectors
    are distinct or shared, and over two calls in a row."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va, P, x = case(name)
    count = 5
    rng = np.random.default_rng(11)
    xs = np.stack([x] + [rng.uniform(-1, 1, n) for _ in range(count - 1)])
    s, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with make_part(n, rp, ci, va, P) as part:
        set_variant(part, variant)
        m = max(n, 1)
        xh = torch.zeros((count, m), dtype=torch.float64).pin_memory()
        xh[:, :n] = torch.from_numpy(xs)
        want = []
        y1 = torch.empty(m, dtype=torch.float64).pin_memory()
        for k in range(count):
            spmv.spmv_apply_host_pipelined(part.h, xh[k], y1, s, s2)
            want.append(y1.numpy()[:n].copy())
        ref0, scale0 = reference(n, rp, ci, va, x)
        assert_fp64_close(want[0], ref0, scale0, "pipelined host path")
        for flags in [0, spmv.HOST_X_BLOCKS, spmv.HOST_Y_PARTS, spmv.HOST_X_BLOCKS | spmv.HOST_Y_PARTS, 0]:
            yh = torch.full((count, m), float("nan"), dtype=torch.float64).pin_memory()
            spmv.spmv_apply_host_many(part.h, count, xh, m, yh, m, flags, s, s2)
            for k in range(count):
                assert np.array_equal(yh[k].numpy()[:n].view(np.uint64), want[k].view(np.uint64)), (flags, k)
        # shared host vectors: the same x every time, every y into one vector
        ys = torch.full((m,), float("nan"), dtype=torch.float64).pin_memory()
        spmv.spmv_apply_host_many(part.h, count, xh[2], 0, ys, 0, 0, s, s2)
        assert np.array_equal(ys.numpy()[:n].view(np.uint64), want[2].view(np.uint64))
        spmv.spmv_apply_host_many(part.h, 0, None, 0, None, 0, 0, s, s2)
        for bad in [dict(count=-1), dict(x_stride=-1), dict(copy=s2), dict(flags=4)]:
            with pytest.raises(spmv.SpmvError) as e:
                spmv.spmv_apply_host_many(part.h, bad.get("count", 2), xh, bad.get("x_stride", m), yh, m,
                                          bad.get("flags", 0), bad.get("copy", s), s2)
            assert e.value.code == spmv.EINVAL
        if n > 1:
            with pytest.raises(spmv.SpmvError) as e:
                spmv.spmv_apply_host_many(part.h, 2, xh, m, yh, 1, 0, s, s2)
            assert e.value.code == spmv.EINVAL


@pytest.mark.parametrize("gran", [0, 1, 2])
@pytest.mark.parametrize("P", [1, 3])
def test_empty_matrix_every_path(gran, P):
    """n = 0: the plan is empty (no rows, entries or halo), and every variant
    family, a random schedule issued eagerly, captured and replayed, the
    host-buffer paths and the index check run without error and write
    nothing (one-element sentinels around them stay as they were)."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    rp = np.zeros(1, np.int64)
    rng = random.Random(5)
    streams = [torch.cuda.Stream() for _ in range(2)]
    x_d = synced(torch.zeros(1, dtype=torch.float64, device="cuda"))
    y_d = synced(torch.full((1,), 7.0, dtype=torch.float64, device="cuda"))
    with make_part(0, rp, np.zeros(0, np.int32), np.zeros(0), P, gran) as part:
        for q in (spmv.Q_N, spmv.Q_NNZ, spmv.Q_NNZ_LOCAL, spmv.Q_NNZ_REMOTE, spmv.Q_N_SEND):
            assert part.query(q) == 0
        dag = E.Dag(part.n_ops, part.dag())
        for v in (("sell", 9), ("sell", 2104), ("vector", 2), ("pairs", 2), ("merge", 0), ("tile", 0),
                  ("warp", 0)):
            set_variant(part, v)
            order, smap = _random_schedule(dag, 2, rng)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            torch.cuda.synchronize()
            spmv.spmv_graph_destroy(part.h, g)
            assert y_d.item() == 7.0 and x_d.item() == 0.0, v
        xh = torch.zeros(1, dtype=torch.float64).pin_memory()
        yh = torch.full((1,), 7.0, dtype=torch.float64).pin_memory()
        spmv.spmv_apply_host_pipelined(part.h, xh, yh, streams[0], streams[1])
        spmv.spmv_apply_host_many(part.h, 3, xh, 0, yh, 0, spmv.HOST_X_BLOCKS, streams[0], streams[1])
        assert yh.item() == 7.0
        assert part.query(spmv.Q_ERROR) == 0
        assert spmv.spmv_part_check(part.h) == 0


# ------------------------------------------------------------------ full sizes
def test_full_size_27pt_150_all_schedules():
    """The 3-D 27-point stencil on 150^3 (n = 3 375 000, 89 915 392 entries),
    P = 4, 2 streams, all 24 schedules captured as graphs: bit-identical y,
    checked in full against the oracle."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va = W.stencil_27pt(150, seed=1)
    assert n == 3375000 and rp[-1] == 448 ** 3
    x = W.uniform_x(n, seed=2)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(2)]
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, 4) as part:
        del ci, va
        assert [part.query(spmv.Q_N_HALO, p) for p in range(4)] == [22650, 45150, 45150, 22650]
        first = None
        for order, smap in E.enumerate_schedules(E.Dag(4, part.dag()), 2):
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
            refill(y_d)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            torch.cuda.synchronize()
            y = y_d.cpu().numpy()
            spmv.spmv_graph_destroy(part.h, g)
            if first is None:
                first = y.copy()
                assert_fp64_close(first, want, scale, "27pt 150^3")
            else:
                assert np.array_equal(y, first)
        assert part.query(spmv.Q_ERROR) == 0


def test_full_size_powerlaw_4M_per_partition():
    """Random power-law matrix, n = 4M, P = 8 per-rank DAG: merge-path and
    thread-per-row products against the oracle in full."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va = W.powerlaw(4_000_000, seed=3)
    x = W.uniform_x(n, seed=4)
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, 8, spmv.PER_PARTITION) as part:
        for variant in (("merge", 0), ("tile", 2)):
            set_variant(part, variant)
            refill(y_d)
            order = [4 * p + k for k in (0, 1, 2, 3) for p in range(8)]
            part.run(order, [0] * 32, [s], x_d, y_d, spmv.RUN_EAGER)
            s.synchronize()
            assert_fp64_close(y_d.cpu().numpy(), want, scale, "powerlaw %s" % (variant,))


def test_full_size_powerlaw_4M_sliced_schedules():
    """The power-law n = 4M, P = 8 per-rank DAG in the form the benchmark
    times: sliced products (LOCAL and REMOTE at several launch shapes, with
    round-robin and cost-balanced CTA ranges, chosen separately), random
    4-stream schedules captured as graphs and
    replayed twice: y bit-identical across variants, schedules and replays,
    and equal to the oracle in full."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va = W.powerlaw(4_000_000, seed=3)
    x = W.uniform_x(n, seed=4)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(4)]
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    rng = random.Random(11)
    first = None
    with make_part(n, rp, ci, va, 8, spmv.PER_PARTITION) as part:
        del ci, va
        dag = E.Dag(part.n_ops, part.dag())
        for lp, rp_ in ((8, 104), (2008, 2104), (2004, 9)):
            part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL, lp)
            part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_SELL, rp_)
            order, smap = _random_schedule(dag, 4, rng)
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
            for _ in range(2):
                refill(y_d)
                part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
                torch.cuda.synchronize()
                y = y_d.cpu().numpy()
                if first is None:
                    first = y.copy()
                    assert_fp64_close(first, want, scale, "powerlaw sliced")
                assert np.array_equal(y.view(np.uint64), first.view(np.uint64)), (lp, rp_)
            spmv.spmv_graph_destroy(part.h, g)
        assert part.query(spmv.Q_ERROR) == 0
        assert spmv.spmv_part_check(part.h) == 0


def test_full_size_powerlaw_4M_relaxed_schedules():
    """The power-law n = 4M, P = 8 per-rank DAG with the sliced products in
    relaxed mode (DAG-only ordering, overlapping independent kernels of one
    stream): random schedules on 1, 2 and 4 streams captured and replayed
    five times each into a NaN-filled y, bit-identical to the stream-ordered
    mode and within the oracle's bound."""
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import schedules as E
    torch = torch_cuda()
    n, rp, ci, va = W.powerlaw(4_000_000, seed=3)
    x = W.uniform_x(n, seed=4)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(4)]
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    rng = random.Random(12)
    with make_part(n, rp, ci, va, 8, spmv.PER_PARTITION) as part:
        del ci, va
        part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL, 2105)
        part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_SELL, 105)
        dag = E.Dag(part.n_ops, part.dag())
        refill(y_d)
        kinds_in_order = [4 * p + k for k in (0, 1, 2, 3) for p in range(8)]   # packs, locals, copies, remotes
        part.run(kinds_in_order, [0] * part.n_ops, streams, x_d, y_d, spmv.RUN_EAGER)
        torch.cuda.synchronize()
        first = y_d.cpu().numpy().copy()
        assert_fp64_close(first, want, scale, "powerlaw strict")
        for ns in (1, 2, 4):
            order, smap = _random_schedule(dag, ns, rng)
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE | spmv.RUN_RELAXED)
            for _ in range(5):
                refill(y_d)
                part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
                torch.cuda.synchronize()
                y = y_d.cpu().numpy()
                assert np.array_equal(y.view(np.uint64), first.view(np.uint64)), ns
            spmv.spmv_graph_destroy(part.h, g)
        assert part.query(spmv.Q_ERROR) == 0


def test_full_size_27pt_150_benchmark_variants():
    """The 27-point stencil 150^3, P = 4, with the products the benchmark
    tunes between: LOCAL in 16-bit-delta or 32-bit sliced form, REMOTE by
    pairs or sliced, round-robin or with balanced CTA ranges; the best
    schedule's shape
    (LOCAL on its own stream) captured and replayed: y equal to the oracle
    in full, and bit-identical across the sliced variants."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    n, rp, ci, va = W.stencil_27pt(150, seed=1)
    x = W.uniform_x(n, seed=2)
    want, scale = reference(n, rp, ci, va, x)
    streams = [torch.cuda.Stream() for _ in range(2)]
    x_d = dev(x)
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    sliced = None
    with make_part(n, rp, ci, va, 4) as part:
        del ci, va
        for (lv, lp), (rv, rpar) in (((spmv.VARIANT_SELL16, 9), (spmv.VARIANT_PAIRS, 1)),
                                     ((spmv.VARIANT_SELL16, 2009), (spmv.VARIANT_SELL, 104)),
                                     ((spmv.VARIANT_SELL, 8), (spmv.VARIANT_SELL, 2004))):
            part.set_op_variant(spmv.OP_LOCAL, lv, lp)
            part.set_op_variant(spmv.OP_REMOTE, rv, rpar)
            order, smap = [0, 2, 1, 3], [0, 1, 0, 0]   # pack, copy, remote on 0; local on 1
            g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
            refill(y_d)
            part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
            torch.cuda.synchronize()
            y = y_d.cpu().numpy()
            spmv.spmv_graph_destroy(part.h, g)
            assert_fp64_close(y, want, scale, "27pt 150^3 %s" % ((lv, lp, rv, rpar),))
            if rv == spmv.VARIANT_SELL:
                # SELL16 and SELL sum every row in the same order
                if sliced is None:
                    sliced = y.copy()
                assert np.array_equal(y.view(np.uint64), sliced.view(np.uint64)), (lv, lp, rv, rpar)
        assert part.query(spmv.Q_ERROR) == 0
        assert spmv.spmv_part_check(part.h) == 0


def test_bounded_wait_reports_timeout_and_context_survives():
    """A wait that nothing completes gives up after its limit and reports
    the timeout status; the device stays usable afterwards."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    assert spmv.spmv_selftest_wait_timeout(2_000_000) == 6
    n, rp, ci, va, P, x = case("lap64")
    want, scale = reference(n, rp, ci, va, x)
    s = torch.cuda.Stream()
    y_d = torch.empty(n, dtype=torch.float64, device="cuda")
    with make_part(n, rp, ci, va, P) as part:
        run_default(part, dev(x), y_d, s)
        s.synchronize()
        assert_fp64_close(y_d.cpu().numpy(), want, scale, "after the timeout self-test")
        assert part.query(spmv.Q_ERROR) == 0


@pytest.mark.parametrize("entry", ["spmv_csr_merge", "spmv_csr_merge_noalloc"])
def test_merge_give_up_path_writes_nothing_outside_y(entry):
    """The merge-path kernel's give-up path (taken when a bounded wait runs
    out), planted from the host: a large product first leaves carries of its
    own rows in the scratch, then a small product gives up from tile 10 on.
    Its error word reads 6, nothing is written past y[n) (where the large
    product's rows would land if a stale carry were used), and the next
    product without the hook is right."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    s = torch.cuda.Stream()
    run = getattr(spmv, entry)
    n0, rp0, ci0, va0 = W.powerlaw(300_000, seed=13)
    big = torch.empty(n0, dtype=torch.float64, device="cuda")
    run(n0, int(rp0[-1]), dev(rp0.astype(np.int32)), dev(ci0), dev(va0), dev(W.uniform_x(n0, seed=1)), big, s)
    s.synchronize()
    assert spmv.spmv_csr_error() == 0
    n, rp, ci, va = W.stencil_27pt(0, seed=14, dims=(20, 20, 20))
    x = W.uniform_x(n, seed=15)
    want, scale = reference(n, rp, ci, va, x)
    tiles = (n + int(rp[-1]) + 2047) // 2048
    assert tiles > 40
    guard = synced(torch.full((n0,), 7.0, dtype=torch.float64, device="cuda"))   # y is guard[:n]
    args = (n, int(rp[-1]), dev(rp.astype(np.int32)), dev(ci), dev(va), dev(x), guard)
    spmv.spmv_selftest_merge_abort(10)
    try:
        run(*args, s)
        s.synchronize()
    finally:
        spmv.spmv_selftest_merge_abort(-1)
    assert spmv.spmv_csr_error() == 6
    g = guard.cpu().numpy()
    assert np.all(g[n:] == 7.0), "a write landed past y[n)"
    run(*args, s)
    s.synchronize()
    assert spmv.spmv_csr_error() == 0
    assert_fp64_close(guard.cpu().numpy()[:n], want, scale, "after the give-up self-test")
    assert np.all(guard.cpu().numpy()[n:] == 7.0)


def test_fp64_probe_does_the_work_it_counts():
    """Every chain of the FP64 probe follows a_{i+1} = m c + a_i, so after k
    steps a_k = a_0 + k m c; the stored sums match that closed form (up to
    k roundings), and the returned count is grid x warps x lanes x 8 chains
    x k."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    k = 1000
    for lanes in (32, 1):
        out = synced(torch.zeros(sms * 2 * 256, dtype=torch.float64, device="cuda"))
        dfma = spmv.spmv_probe_dfma(k, 2, lanes, out, out.numel(), None)
        torch.cuda.synchronize()
        assert dfma == sms * 2 * 8 * lanes * 8 * k
        o = out.cpu().numpy().reshape(-1, 32)
        gid = np.arange(o.size).reshape(-1, 32)
        m, c = 1e-3, 1e-3
        a0 = 1.0 + 1e-3 * np.arange(8)[None, None, :] + 1e-9 * (gid & 1023)[:, :, None]
        run = a0 + k * (m * c)
        want = np.where((np.arange(32) < lanes)[None, :, None], run, a0).sum(axis=2)
        assert np.allclose(o, want, rtol=1e-12, atol=0)
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_probe_dfma(10, 2, 32, out, 10, None)
    assert e.value.code == spmv.EINVAL


def test_gather_probe_sums_what_it_gathers():
    """Thread g of the gather probe sums table[idx[k]] for k = g mod T: the
    stored sums equal numpy's over the same positions (up to rounding)."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    T = sms * 2 * 256
    rng = np.random.default_rng(21)
    table = rng.uniform(-1, 1, 1 << 20)
    count = 9 * T + 12345   # a ragged tail after the four-in-flight rounds
    idx = rng.integers(0, table.size, count).astype(np.int32)
    out = synced(torch.zeros(T, dtype=torch.float64, device="cuda"))
    spmv.spmv_probe_gather(dev(table), dev(idx), count, 2, out, T, None)
    torch.cuda.synchronize()
    vals = np.zeros(10 * T)
    vals[:count] = table[idx]
    want = vals.reshape(10, T).sum(axis=0)
    assert np.allclose(out.cpu().numpy(), want, rtol=0, atol=1e-12)


def test_merge_abort_hook_rejects_bad_tiles():
    from paper_2203_02530_gb300 import spmv
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_selftest_merge_abort(-2)
    assert e.value.code == spmv.EINVAL


_PLAIN_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2203_02530_gb300 import spmv, workloads as W
n, rp, ci, va = W.powerlaw(3000, seed=3, cap=500)
x = W.uniform_x(n, seed=99)
s = [torch.cuda.Stream() for _ in range(2)]
x_d = torch.from_numpy(x).cuda()
y_d = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
torch.cuda.synchronize()
with spmv.Part(n, rp, ci, va, 3, spmv.PER_PARTITION) as part:
    part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL, 2008)
    part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_MERGE, 0)
    order = [4 * p + k for k in (0, 1, 2, 3) for p in range(3)]
    g = part.run(order, [0, 1] * 6, s, x_d, y_d, spmv.RUN_CAPTURE)
    part.run(order, [0, 1] * 6, s, x_d, y_d, spmv.RUN_REPLAY, g)
    torch.cuda.synchronize()
np.save(sys.argv[2], y_d.cpu().numpy())
"""


@pytest.mark.parametrize("no_pdl", ["1", "0"])
def test_programmatic_launch_off_and_on_give_the_same_y(tmp_path, no_pdl):
    """The same captured per-rank schedule (sliced and merge-path products,
    two streams) in a child process with programmatic dependent launch
    switched off (SPMV_NO_PDL=1) or left on gives this process's y bit for
    bit."""
    import os
    import subprocess
    import sys
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "y.npy")
    env = dict(os.environ, SPMV_NO_PDL=no_pdl)
    subprocess.run([sys.executable, "-c", _PLAIN_CHILD, root, out], env=env, check=True, timeout=600)
    n, rp, ci, va = W.powerlaw(3000, seed=3, cap=500)
    x = W.uniform_x(n, seed=99)
    want, scale = reference(n, rp, ci, va, x)
    s = [torch.cuda.Stream() for _ in range(2)]
    x_d = dev(x)
    y_d = synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))
    with make_part(n, rp, ci, va, 3, spmv.PER_PARTITION) as part:
        part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL, 2008)
        part.set_op_variant(spmv.OP_REMOTE, spmv.VARIANT_MERGE, 0)
        order = [4 * p + k for k in (0, 1, 2, 3) for p in range(3)]
        g = part.run(order, [0, 1] * 6, s, x_d, y_d, spmv.RUN_CAPTURE)
        part.run(order, [0, 1] * 6, s, x_d, y_d, spmv.RUN_REPLAY, g)
        torch.cuda.synchronize()
    y = y_d.cpu().numpy()
    assert_fp64_close(y, want, scale, "programmatic launch")
    assert np.array_equal(np.load(out).view(np.uint64), y.view(np.uint64))


def test_index_check_finds_the_planted_indices():
    """The plan checks' kernels count exactly the two planted out-of-range
    indices of their self-test (nothing is dereferenced)."""
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    assert spmv.spmv_selftest_check() == 2


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("gran", [0, 1])
def test_every_plan_index_in_range(name, gran):
    """Every index array of every plan (CSR blocks, halo maps, send lists,
    pack positions, and the sliced layouts with their 16-bit deltas once
    built) lies inside the range its definition allows."""
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    n, rp, ci, va, P, x = case(name)
    with make_part(n, rp, ci, va, P, gran) as part:
        assert spmv.spmv_part_check(part.h) == 0
        part.set_variant(spmv.VARIANT_SELL, 4)
        assert spmv.spmv_part_check(part.h) == 0
        try:
            part.set_op_variant(spmv.OP_LOCAL, spmv.VARIANT_SELL16, 2009)
        except spmv.SpmvError as e:
            assert e.code == spmv.EINVAL    # some |column - row| needs more than 16 bits
        assert spmv.spmv_part_check(part.h) == 0
