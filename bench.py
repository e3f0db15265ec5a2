#!/usr/bin/env python
"""Benchmark of the row-partitioned FP64 SpMV hot path on one GB300.

Workload: 3-D 27-point stencil on 150^3 (n = 3 375 000, 89 915 392 entries,
values U[-1,1] with diagonal 27, seeds 1 and 2), P = 4 virtual ranks, 2
streams.  Every valid schedule of the pack / local / copy / remote DAG is
enumerated (24) and captured as a CUDA graph; each is measured with the
paper's protocol (samples repeated for 0.01 s, Sec. III-C.3) and the fastest
is the one timed.  A step is one replay of that graph: one whole SpMV.

Output: one JSON line (rank 0).  ``value`` is effective GB/s = algorithmic
bytes per SpMV x steps / time, summed over ranks (each rank runs its own
replica: weak scaling, no data-path collective).  On one GPU the line also
carries the metric's other configurations as sub-objects, each measured in
the same run with its own value, roofline, latency, end-to-end figure, CPU
baseline and clocks: ``powerlaw`` (n = 4M power-law rows, P = 8 per-rank
DAG, a bounded MCTS search), ``batched`` (256 matrices in one persistent
launch against each matrix through the tuned single-matrix product) and
``serving`` (Poisson arrivals served with continuous batching against one
plain launch per request).  ``--impl reference`` times the CPU oracle on the
host cores instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV effective GB/s (% HBM peak), batched/served vs plain; p50/p99 latency"
WORKLOAD = "27-point stencil 150^3 (n=3375000, nnz=89915392), P=4 row blocks, 2 streams, best of 24 schedules"
FALLBACK_HBM = 6800.0


# ---------------------------------------------------------------- ranks
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(dist, value, device=None):
    """Largest value over ranks (barrier included)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None, period_ms=100):
        self.uuid = uuid
        self.period_ms = period_ms
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [c.strip() for c in line.split(",")]
                if len(f) < 9:
                    continue
                if self.uuid and self.uuid not in f[0] and f[0] not in self.uuid:
                    continue
                rows.append(f)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3])] or [0.0])}


def clocks_rejected(c):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(c.get("reasons", [])):
        return True
    if c.get("sm_mhz") and c.get("sm_max_mhz") and c["sm_mhz"] < 0.6 * c["sm_max_mhz"] \
            and "sw_power_cap" not in c.get("reasons", []):
        return True
    return False


# ---------------------------------------------------------------- peaks
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM, "fallback"


# the files each profiled kernel is built from (besides the shared headers)
KERNEL_FILES = {"csr_sell_kernel": ["sell.cu"], "merge_kernel": ["merge.cu"],
                "batch_sliced_persistent_kernel": ["batch.cu", "batch.h"],
                "batch_persistent_kernel": ["batch.cu", "batch.h"]}
SHARED_HEADERS = ["internal.h", "pdl.cuh"]


def kernel_source_hash(kernel):
    """Hash of the code a kernel is built from (comments and blank lines
    left out, so that a comment edit does not invalidate a profile)."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_FILES.get(kernel, ["kernels.cu"]) + SHARED_HEADERS:
        with open(os.path.join(ROOT, "paper_2203_02530_gb300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(workload, key):
    """DRAM bytes per launch (or per launch group) of `key` (kernel/variant/
    param) on `workload` from the committed ncu summary, if it was taken on
    the kernel's current sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    k = d.get("workloads", {}).get(workload, {}).get(key)
    if k is None or k.get("source_hash") != kernel_source_hash(key.split("/")[0]):
        return None
    return k.get("dram_bytes_per_full_launch")


def fp64_probe(dev, props, seconds=0.25):
    """Measured FP64 FMA throughput of this GPU (the library's DFMA probe,
    timed with CUDA events, SM clock sampled meanwhile): the best G DFMA/s
    over 1, 2, 4 and 8 CTAs of 256 threads per SM with 32 active lanes per
    warp, and the same launch with 1 active lane per warp."""
    import torch
    from paper_2203_02530_gb300 import benchmark, spmv
    s = torch.cuda.Stream(device=dev)
    cap = props.multi_processor_count * 8 * 256
    out = torch.empty(cap, dtype=torch.float64, device=dev)

    def rate(cps, lanes, budget):
        iters = 1 << 10
        while True:   # size one launch to about 10 ms
            t = benchmark.time_loop(lambda: spmv.spmv_probe_dfma(iters, cps, lanes, out, cap, s), s, 1, warmup=1)
            if t > 0.01 or iters >= 1 << 30:
                break
            iters *= 2
        reps = max(2, int(budget / t))
        dfma = spmv.spmv_probe_dfma(iters, cps, lanes, out, cap, s)
        t = benchmark.time_loop(lambda: spmv.spmv_probe_dfma(iters, cps, lanes, out, cap, s), s, reps, warmup=1)
        return dfma / t, iters, reps

    sampler = ClockSampler(uuid=str(getattr(props, "uuid", "")) or None)
    sampler.start()
    sweep = {cps: rate(cps, 32, seconds / 5) for cps in (1, 2, 4, 8)}
    best = max(sweep, key=lambda c: sweep[c][0])
    one = rate(best, 1, seconds / 5)
    clocks = sampler.stop()
    mhz = clocks.get("sm_mhz") or props.clock_rate / 1e3
    r = sweep[best][0]
    return {"dfma_per_s": r, "unit": "G DFMA/s", "g_dfma_per_s": round(r / 1e9, 1),
            "per_clk_per_sm": round(r / (mhz * 1e6) / props.multi_processor_count, 3),
            "sm_mhz": mhz, "ctas_per_sm": best,
            "sweep_g_dfma_per_s": {str(c): round(v[0] / 1e9, 1) for c, v in sorted(sweep.items())},
            "one_lane_g_warp_instr_per_s": round(one[0] / 1e9, 2),
            "full_warp_g_warp_instr_per_s": round(r / 32 / 1e9, 2),
            "how": "spmv_probe_dfma: 1, 2, 4 and 8 CTAs x 256 threads per SM, 8 chains of DFMAs per lane, "
                   "each launch about 10 ms, CUDA events; the best is the peak; the one-lane run keeps 1 lane "
                   "of each warp busy at the best CTA count"}


def gather_probe(dev, props, table_len=4_000_000, count=1 << 26, seconds=0.2):
    """Measured rate of scattered 8-byte reads (the library's gather probe,
    CUDA events): `count` uniformly random positions into a table of
    `table_len` doubles (32 MB: L2-resident, the size of the power-law x),
    read through a coalesced int32 index stream as a product reads its
    columns.  Returns G gathers/s."""
    import torch
    from paper_2203_02530_gb300 import benchmark, spmv
    s = torch.cuda.Stream(device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(31)
    table = torch.rand(table_len, dtype=torch.float64, device=dev, generator=gen)
    idx = torch.randint(0, table_len, (count,), dtype=torch.int32, device=dev, generator=gen)
    # the table and indices come from the current stream; the probe runs on s
    torch.cuda.synchronize(dev)
    cps = 4
    cap = props.multi_processor_count * cps * 256
    out = torch.empty(cap, dtype=torch.float64, device=dev)
    run = lambda: spmv.spmv_probe_gather(table, idx, count, cps, out, cap, s)
    t = benchmark.time_loop(run, s, 1, warmup=2)
    reps = max(3, int(seconds / t))
    t = benchmark.time_loop(run, s, reps, warmup=1)
    del table, idx, out
    return {"g_gathers_per_s": round(count / t / 1e9, 2), "table_mb": round(table_len * 8 / 1e6, 1),
            "how": "spmv_probe_gather: %d uniformly random 8-byte reads from a %d-entry table through a "
                   "coalesced int32 index stream, %d CTAs x 256 threads, 4 in flight per thread, CUDA events "
                   "over %d launches" % (count, table_len, props.multi_processor_count * cps, reps)}


# ---------------------------------------------------------------- workload
def workload(seed_a=1, seed_x=2, g=150):
    from paper_2203_02530_gb300 import workloads as W
    n, rp, ci, va = W.stencil_27pt(g, seed=seed_a)
    x = W.uniform_x(n, seed=seed_x)
    return n, rp, ci, va, x


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(n, rp, ci, va, x, P, seconds):
    """Time the oracle's partitioned SpMV (single thread) for about
    `seconds`; returns (GB/s, reps, seconds, alg_bytes)."""
    import oracle
    pl = oracle.OraclePlan(n, rp, ci, va, P)
    nnz = int(rp[-1] - rp[0])
    nnz_r = sum(len(pl.export(oracle.R_COL, p)) for p in range(P))
    nsend = len(pl.export(oracle.SEND_IDX))
    rr = 0
    for p in range(P):
        r = pl.export(oracle.R_PTR, p)
        rr += int((r[1:] > r[:-1]).sum())
    alg = cpu_alg_bytes(n, nnz - nnz_r, nnz_r, rr, nsend)
    pl.spmv(x)   # warm
    reps, t0 = 0, time.perf_counter()
    while True:
        pl.spmv(x)
        reps += 1
        t = time.perf_counter() - t0
        if t >= seconds:
            break
    pl.close()
    return alg * reps / t / 1e9, reps, t, alg


def oracle_parallel_rate(n, rp, ci, va, x, seconds):
    """The oracle's plain product (the definition, unpartitioned) with its
    rows shared among all host threads, timed for about `seconds`."""
    import oracle
    nnz = int(rp[-1] - rp[0])
    alg = 12 * nnz + 4 * (n + 1) + 16 * n
    oracle.csr_spmv_rows_parallel(n, rp, ci, va, x)   # warm
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.csr_spmv_rows_parallel(n, rp, ci, va, x)
        reps += 1
        t = time.perf_counter() - t0
        if t >= seconds:
            break
    return {"value": round(alg * reps / t / 1e9, 3), "unit": "GB/s", "cores": oracle.max_threads(),
            "kind": "oracle", "sample": "%d plain CSR products (rows split over OpenMP threads) of the same "
                                        "matrix in %.1f s" % (reps, t)}


def cpu_alg_bytes(n, nnz_l, nnz_r, n_rr, n_send):
    # the same counting as the library: local entries, row pointers, x, y;
    # remote entries, its compressed rows and y update; pack, exchange, halo
    b = 12 * nnz_l + 4 * (n + 1) + 8 * n + 8 * n
    b += 12 * nnz_r + 4 * (n_rr + 1) + 4 * n_rr + 16 * n_rr
    b += 12 * n_send + 16 * n_send + 8 * n_send
    return b


# ---------------------------------------------------------------- our arm
WORKLOADS = {
    # name: (description, generator, P, streams, granularity, search)
    "stencil27": (WORKLOAD, lambda: workload(), 4, 2, 0, "exhaustive"),
    "laplacian": ("5-point Laplacian 64x64 (n=4096, nnz=20224), P=2, 1 stream, the default "
                  "schedule (pack, local, copy, remote); L2-resident: replay latency",
                  lambda: laplacian(), 2, 1, 0, "fixed"),
    "powerlaw": ("random power-law n=4M (Zipf(2) row lengths, cap 4096; 80% of columns within "
                 "+-n/8), P=8 per-rank DAG (32 ops), 4 streams, MCTS-sampled schedules",
                 lambda: powerlaw(), 8, 4, 1, "mcts"),
    "band": ("the paper's band matrix: 150000 x 150000, 1.5M entries uniform in |i-j| <= 37500, "
             "P=4, 2 streams, all 24 schedules; L2-resident (replay latency)",
             lambda: band(), 4, 2, 0, "exhaustive"),
    "stencil27_segments": ("27-point stencil 150^3 (n=3375000, nnz=89915392), P=4, per-segment DAG "
                           "(LOCAL and REMOTE per rank, PACK and COPY per halo segment: 20 ops), "
                           "2 streams, MCTS-sampled schedules",
                           lambda: workload(), 4, 2, 2, "mcts"),
}


def band():
    from paper_2203_02530_gb300 import workloads as W
    n, rp, ci, va = W.band(150_000, 1_500_000, 37_500, seed=7)
    return n, rp, ci, va, W.uniform_x(n, seed=8)


def laplacian():
    from paper_2203_02530_gb300 import workloads as W
    n, rp, ci, va = W.laplacian_5pt(64)
    return n, rp, ci, va, W.uniform_x(n, seed=0)


def powerlaw():
    from paper_2203_02530_gb300 import workloads as W
    n, rp, ci, va = W.powerlaw(4_000_000, seed=3)
    return n, rp, ci, va, W.uniform_x(n, seed=4)


_DIST = {}


def dist_once(world):
    if "d" not in _DIST:
        _DIST["d"] = dist_init(world, "nccl")
    return _DIST["d"]


def per_sample_latency(step, stream, count):
    """Per-sample times (s) of `count` back-to-back samples, each bracketed
    by its own pair of CUDA events on `stream`."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(count + 1)]
    ev[0].record(stream)
    for i in range(count):
        step()
        ev[i + 1].record(stream)
    ev[-1].synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) * 1e-3 for i in range(count)]


def latency_block(per_sample, meas):
    from paper_2203_02530_gb300 import benchmark
    return {"p50": round(benchmark.percentile(per_sample, 50) * 1e6, 2),
            "p99": round(benchmark.percentile(per_sample, 99) * 1e6, 2),
            "samples": len(per_sample), "protocol": "per sample: CUDA events around each of back-to-back "
                                                    "replays",
            "measurements": {"p50": round(benchmark.percentile(meas, 50) * 1e6, 2),
                             "p99": round(benchmark.percentile(meas, 99) * 1e6, 2),
                             "count": len(meas), "protocol": "Sec. III-C.3: mean over 0.01 s of samples each"}}


def run_ours(args, world, rank, local, fp64=None):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = dist_once(world)
    from paper_2203_02530_gb300 import autotune, benchmark, search, spmv

    desc, gen, P, S, gran, mode = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    n, rp, ci, va, x = gen()
    part = spmv.Part(n, rp, ci, va, P, gran)
    x_d = torch.from_numpy(x).to(dev)
    y_d = torch.empty(n, dtype=torch.float64, device=dev)
    streams = [torch.cuda.Stream(device=dev) for _ in range(S)]
    sig = autotune.signature(n, rp, P, props.name)
    tuned = autotune.tune(part, x_d, y_d, streams[0], sig=sig, use_cache=not args.retune)
    variant, vparam = tuned["local"]
    tune_times = tuned["times"]
    # with both products on the sliced layout the CSR copy is a second copy
    # of the matrix that no product reads: release it
    plan_bytes = {"tuned": part.query(spmv.Q_DEVICE_BYTES)}
    if variant in (spmv.VARIANT_SELL, spmv.VARIANT_SELL16) and tuned["remote"][0] == spmv.VARIANT_SELL:
        part.release_csr()
    plan_bytes["timed"] = part.query(spmv.Q_DEVICE_BYTES)

    # the design space: every schedule (coarse DAG), MCTS samples (per-rank
    # DAG) or the single default order
    rec = search.Recorder(args.records, meta={"workload": args.workload}) if args.records else None
    if args.records:
        with open(args.records + ".dag.json", "w") as f:
            json.dump({"n_ops": part.n_ops, "edges": part.dag(), "P": P, "streams": S,
                       "names": part.op_names()}, f)
    search_cmp = None
    t_search = time.perf_counter()
    # the design space searched in each ordering mode: "strict" runs the
    # kernels of a stream one after another (the paper's semantics),
    # "relaxed" orders them by the DAG alone (SPMV_RUN_RELAXED), "defer" lets
    # remote products sum their rows before waiting for the kernel before
    # them (SPMV_RUN_DEFER)
    by_mode = {}
    for run_mode in args.run_modes.split(","):
        strict = run_mode == "strict"
        rec_m = rec if (rec is not None and strict) else None
        # the minimum of a few 0.01 s measurements per program, so that a host
        # hiccup during one measurement does not masquerade as a slow program
        evaluate = search.graph_evaluator(part, streams, x_d, y_d, recorder=rec_m, measurements=3
                                          if mode == "exhaustive" else 2, relaxed="relaxed" in run_mode,
                                          defer="defer" in run_mode)
        if mode == "exhaustive":
            sched = search.exhaustive(part, streams, evaluate)
        elif mode == "mcts":
            # the sample budget is split over the orderings searched
            n_modes = len(args.run_modes.split(","))
            sched, _ = search.mcts(part, streams, evaluate, -(-args.mcts_iters // n_modes), seed=0)
            if args.random_baseline and strict:
                cmp = {"samples": args.random_baseline}
                mt = [r[2] for r in sched[:args.random_baseline]]
                cmp["mcts"] = {"best_us": round(min(mt) * 1e6, 2), "worst_us": round(max(mt) * 1e6, 2)}
                for rmode in ("uniform", "per_decision"):
                    rand = search.random_sampling(part, streams, evaluate, args.random_baseline, seed=1,
                                                  mode=rmode)
                    rt = [r[2] for r in rand]
                    cmp["random_" + rmode] = {"best_us": round(min(rt) * 1e6, 2),
                                              "worst_us": round(max(rt) * 1e6, 2), "samples": len(rand)}
                search_cmp = cmp
        else:
            order = list(range(part.n_ops))
            sched = [(order, [0] * part.n_ops, evaluate(order, [0] * part.n_ops))]
        by_mode[run_mode] = sorted(sched, key=lambda r: r[2])
    run_mode = min(by_mode, key=lambda m: by_mode[m][0][2])
    sched = by_mode[run_mode]
    mode_flag = {"strict": 0, "relaxed": spmv.RUN_RELAXED, "defer": spmv.RUN_DEFER,
                 "relaxed+defer": spmv.RUN_RELAXED | spmv.RUN_DEFER}[run_mode]
    order, smap, t_best = sched[0]
    # the variants were tuned on launches timed one after another; a program
    # overlaps its kernels (a per-rank program its ranks', a deferred remote
    # product the local product's tail), so the best program is re-timed with
    # the three fastest LOCAL x three fastest REMOTE variants of the tuning and
    # the fastest pair kept
    in_context = None
    if len(sched[0][0]) > 1:
        def top(op):
            c = sorted(((t, v, p) for (o, v, p), t in tune_times.items() if o == op))
            return [(v, p) for _, v, p in c[:3]]
        ev_ctx = search.graph_evaluator(part, streams, x_d, y_d, measurements=3, relaxed="relaxed" in run_mode,
                                        defer="defer" in run_mode)
        in_context = {}
        best = (t_best, tuple(tuned["local"]), tuple(tuned["remote"]))
        for lv in top(spmv.OP_LOCAL):
            for rv in top(spmv.OP_REMOTE):
                try:
                    part.set_op_variant(spmv.OP_LOCAL, *lv)
                    part.set_op_variant(spmv.OP_REMOTE, *rv)
                except spmv.SpmvError:
                    continue
                t = ev_ctx(order, smap)
                in_context["%d,%d/%d,%d" % (lv + rv)] = round(t * 1e6, 2)
                if t < best[0]:
                    best = (t, lv, rv)
        part.set_op_variant(spmv.OP_LOCAL, *best[1])
        part.set_op_variant(spmv.OP_REMOTE, *best[2])
        tuned = dict(tuned, local=best[1], remote=best[2])
        variant, vparam = tuned["local"]
        t_best = best[0]
        # a CSR variant timed here rebuilt the CSR copy: release it again when
        # both kept products are sliced
        if variant in (spmv.VARIANT_SELL, spmv.VARIANT_SELL16) and tuned["remote"][0] == spmv.VARIANT_SELL:
            try:
                part.release_csr()
            except spmv.SpmvError as e:   # reported through the plan bytes; the products are unaffected
                print("CSR copy kept: %s" % e, file=sys.stderr)
        plan_bytes["timed"] = part.query(spmv.Q_DEVICE_BYTES)
    t_search = time.perf_counter() - t_search
    spread = sched[-1][2] / sched[0][2]
    g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE | mode_flag)
    step = lambda: part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
    part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)   # counts the launches of a step
    launches_per_step = part.query(spmv.Q_LAST_LAUNCHES)
    alg = part.query(spmv.Q_ALG_BYTES)
    alg_local = part.query(spmv.Q_ALG_BYTES_LOCAL)
    nnz_l = part.query(spmv.Q_NNZ_LOCAL)

    def timed_region():
        # the clock sampler starts (and settles) before the warm-up, so that
        # the warm-up steps run right before the timed ones and the GPU is not
        # left idle between them
        sampler = ClockSampler(uuid=str(getattr(props, "uuid", "")) or None)
        sampler.start()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_region")
        e0.record(streams[0])
        for _ in range(args.steps):
            step()
        e1.record(streams[0])
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1) * 1e-3, clocks

    elapsed, clocks = timed_region()
    remeasured = False
    if clocks_rejected(clocks):
        elapsed, clocks = timed_region()
        remeasured = True
    elapsed = max_over_ranks(dist, elapsed, dev)
    value = world * alg * args.steps / elapsed / 1e9

    # the dominant kernel (the LOCAL product) timed alone on the stream the
    # schedule launches it on, with CUDA events: one launch over all ranks
    # for a coarse plan, the P per-rank launches in a row for a per-rank plan
    # (the launches its schedules run)
    per_rank = gran != spmv.COARSE
    s_local = streams[smap[spmv.OP_LOCAL]] if not per_rank else streams[0]
    if per_rank:
        local_unit = lambda: [spmv.spmv_local(part.h, p, x_d, y_d, s_local) for p in range(P)]
    else:
        local_unit = lambda: spmv.spmv_local(part.h, -1, x_d, y_d, s_local)
    t_local = benchmark.time_loop(local_unit, s_local, max(50, min(args.steps, 1000)))
    peak, peak_kind = hbm_peak()
    achieved = alg_local / t_local / 1e9
    kname = {spmv.VARIANT_TILE: "csr_tile_kernel", spmv.VARIANT_VECTOR: "csr_vector_kernel",
             spmv.VARIANT_MERGE: "merge_kernel", spmv.VARIANT_PAIRS: "csr_pair_kernel",
             spmv.VARIANT_WARP: "csr_warp_kernel", spmv.VARIANT_SELL: "csr_sell_kernel",
             spmv.VARIANT_SELL16: "csr_sell_kernel"}[variant]
    traffic = profiled_traffic(args.workload, "%s/%d/%d" % (kname, variant, vparam))

    # latency of the best schedule: per sample, and per 0.01 s measurement
    per_sample = per_sample_latency(step, streams[0], max(args.latency_samples, args.steps))
    meas = benchmark.measurements(step, streams[0], args.measurements)

    # end to end through the C ABI with host buffers
    xi, yi = spmv.spmv_part_io_buffers(part.h)
    ge = part.run(order, smap, streams, xi, yi, spmv.RUN_CAPTURE | mode_flag)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(n, dtype=torch.float64).pin_memory()
    for _ in range(3):
        spmv.spmv_apply_host(part.h, ge, xh, yh, streams[0])
    k_e2e = max(10, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        spmv.spmv_apply_host(part.h, ge, xh, yh, streams[0])
    t_e2e_graph = max_over_ranks(dist, (time.perf_counter() - t0) / k_e2e, dev)
    # the same through the pipelined host path (x block transfers overlapped
    # with the LOCAL products; variants as tuned)
    cs = torch.cuda.Stream()
    for _ in range(3):
        spmv.spmv_apply_host_pipelined(part.h, xh, yh, cs, streams[0])
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        spmv.spmv_apply_host_pipelined(part.h, xh, yh, cs, streams[0])
    t_e2e = max_over_ranks(dist, (time.perf_counter() - t0) / k_e2e, dev)
    # a stream of independent products through host buffers (the same x sent
    # and the same y returned every step): product k+1's x goes in while
    # product k computes and its y comes out
    # with the copies' granularity (x in rank blocks or in one copy, y out in
    # parts or in one copy) chosen by a short sweep
    many_flags = {"x whole, y whole": 0, "x blocks, y whole": spmv.HOST_X_BLOCKS,
                  "x whole, y parts": spmv.HOST_Y_PARTS,
                  "x blocks, y parts": spmv.HOST_X_BLOCKS | spmv.HOST_Y_PARTS}
    many_sweep = {}
    for name, fl in many_flags.items():
        spmv.spmv_apply_host_many(part.h, 3, xh, 0, yh, 0, fl, cs, streams[0])
        t0 = time.perf_counter()
        spmv.spmv_apply_host_many(part.h, 20, xh, 0, yh, 0, fl, cs, streams[0])
        many_sweep[name] = max_over_ranks(dist, (time.perf_counter() - t0) / 20, dev)
    many_best = min(many_sweep, key=many_sweep.get)
    t0 = time.perf_counter()
    spmv.spmv_apply_host_many(part.h, k_e2e, xh, 0, yh, 0, many_flags[many_best], cs, streams[0])
    t_e2e_many = max_over_ranks(dist, (time.perf_counter() - t0) / k_e2e, dev)
    e2e_paths = {"spmv_apply_host_many": t_e2e_many, "spmv_apply_host_pipelined": t_e2e,
                 "spmv_apply_host": t_e2e_graph}
    e2e_best = min(e2e_paths, key=e2e_paths.get)
    # where the end-to-end time goes: the host link alone, each direction and
    # both at once (x in on one stream while y goes out on another)
    xb_d = torch.empty(n, dtype=torch.float64, device=dev)
    yb_d = torch.empty(n, dtype=torch.float64, device=dev)
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def link(which):
        if which in ("in", "both"):
            with torch.cuda.stream(s_in):
                xb_d.copy_(xh, non_blocking=True)
        if which in ("out", "both"):
            with torch.cuda.stream(s_out):
                yh.copy_(yb_d, non_blocking=True)
        s_in.synchronize()
        s_out.synchronize()

    link_us = {}
    for which in ("in", "out", "both"):
        link(which)
        t0 = time.perf_counter()
        for _ in range(20):
            link(which)
        link_us[which] = round((time.perf_counter() - t0) / 20 * 1e6, 1)
    err = part.query(spmv.Q_ERROR)
    dev_bytes = part.query(spmv.Q_DEVICE_BYTES)   # with the host paths' device vectors

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, reps, secs, _ = oracle_rate(n, rp, ci, va, x, P, args.cpu_seconds)
        cpu = {"value": round(rate, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "%d full partitioned SpMVs of the same matrix (P=%d) in %.1f s, "
                         "single-threaded C oracle on the host cores (nproc=%d)" % (
                             reps, P, secs, os.cpu_count() or 0)}
        cpu["all_cores"] = oracle_parallel_rate(n, rp, ci, va, x, args.cpu_seconds / 2)
    part.close()
    if rank != 0:
        return None
    if fp64 is None:
        fp64 = fp64_probe(dev, props)
    dfma_rate = nnz_l / t_local
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed / args.steps * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "n": n, "nnz": int(rp[-1]), "P": P, "streams": S,
                   "granularity": ("coarse", "per-rank", "per-segment")[gran],
                   "search": mode, "schedules_measured": sum(len(v) for v in by_mode.values()),
                   "search_seconds": round(t_search, 1), "ordering": run_mode,
                   "best_us_by_ordering": {m: round(v[0][2] * 1e6, 2) for m, v in by_mode.items()},
                   "variants_in_context_us": in_context,
                   "best_order": order, "best_streams": smap,
                   "variant": {"local": list(tuned["local"]), "remote": list(tuned["remote"])},
                   "l2": "inputs larger than L2" if 12 * int(rp[-1]) > 129e6
                         else "L2-resident (replay latency)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "alg_bytes_per_step": alg, "plan_device_bytes": plan_bytes["timed"],
                   "plan_device_bytes_before_csr_release": plan_bytes["tuned"],
                   "plan_device_bytes_with_host_vectors": dev_bytes},
        "percent_hbm": round(100.0 * value / world / peak, 2),
        "roofline": dict({"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                          "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                          "traffic": traffic, "peak_kind": peak_kind,
                          "alg_bytes_per_launch": alg_local, "launch_us": round(t_local * 1e6, 2),
                          "launches": P if per_rank else 1},
                         **({} if traffic is None else {
                             "dram_gbs": round(traffic / t_local / 1e9, 1),
                             "dram_frac": round(traffic / t_local / 1e9 / peak, 4),
                             "note": "achieved counts the CSR algorithmic bytes; the DRAM traffic of "
                                     "the launch (ncu) is `traffic`"})),
        "fp64": {"dfma_per_s": round(dfma_rate / 1e9, 1), "unit": "G DFMA/s",
                 "peak": fp64["g_dfma_per_s"], "frac": round(dfma_rate / fp64["dfma_per_s"], 4),
                 "peak_kind": "measured by spmv_probe_dfma in this run (%.3f DFMA/clk/SM at %.0f MHz)" % (
                     fp64["per_clk_per_sm"], fp64["sm_mhz"]),
                 "note": "one DFMA per stored local entry over the LOCAL launch time"},
        "gather": None if "gather" not in fp64 else {
            "achieved": round(nnz_l / t_local / 1e9, 2), "unit": "G gathers/s",
            "peak": fp64["gather"]["g_gathers_per_s"],
            "frac": round(nnz_l / t_local / 1e9 / fp64["gather"]["g_gathers_per_s"], 4),
            "note": "one x gather per stored local entry over the LOCAL launch time, against the gather "
                    "probe's rate for random reads from an L2-resident table"},
        "latency_us": latency_block(per_sample, meas),
        "schedule_spread": round(spread, 4),
        "search_vs_random": search_cmp,
        "e2e": {"value": round(alg / e2e_paths[e2e_best] / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                "ms_per_step": round(e2e_paths[e2e_best] * 1e3, 4),
                "path": e2e_best,
                "paths": {k: {"value": round(alg / v / 1e9, 2), "ms_per_step": round(v * 1e3, 4)}
                          for k, v in e2e_paths.items()},
                "paths_note": "spmv_apply_host and spmv_apply_host_pipelined: one product per call, "
                              "returning after y arrived (the latency of one end-to-end product); "
                              "spmv_apply_host_many: %d independent products in one call, consecutive "
                              "ones overlapped (x of the next in while y of the last goes out)" % k_e2e,
                "many_copies": many_best,
                "many_sweep_us": {k: round(v * 1e6, 1) for k, v in many_sweep.items()},
                "vs_device_step": ("the streamed products ran faster than the device-timed step: there "
                                   "each graph replay starts after the previous one ends (the paper's "
                                   "protocol), while consecutive streamed products overlap, each one's "
                                   "kernels filling the previous one's ramps and tails"
                                   if e2e_paths[e2e_best] < elapsed / args.steps else None),
                "breakdown_us": {"x_in_alone": link_us["in"], "y_out_alone": link_us["out"],
                                 "in_and_out_together": link_us["both"],
                                 "device_step": round(elapsed / args.steps * 1e6, 1),
                                 "note": "host-timed pinned copies of x (in) and y (out), %d bytes each; the "
                                         "pipelined path overlaps both with the products" % (8 * n)}},
        "cpu_baseline": cpu,
        "clocks": clocks, "remeasured": remeasured,
        "gpu_launches": launches_per_step * args.steps,
        "device_error_word": err,
        "autotune_us": {"%s %d,%d" % ("local" if k[0] == spmv.OP_LOCAL else "remote", k[1], k[2]):
                        round(v * 1e6, 1) for k, v in tune_times.items()},
    }
    return line


# ---------------------------------------------------------------- batched
# variants the plain per-matrix form picks from, per matrix (the families the
# single-matrix tuner chooses on stencils, Zipf rows and skewed rows)
def plain_candidates():
    from paper_2203_02530_gb300 import spmv
    return [(spmv.VARIANT_SELL16, 107), (spmv.VARIANT_SELL16, 9), (spmv.VARIANT_SELL, 105),
            (spmv.VARIANT_SELL, 8), (spmv.VARIANT_SELL, 2105), (spmv.VARIANT_SELL, 4),
            (spmv.VARIANT_VECTOR, 2), (spmv.VARIANT_MERGE, 0)]


def plain_per_matrix(mats, offs, x_d, s, reps=10):
    """The plain form of many products: every matrix through the library's
    single-matrix product (a plan with P = 1, whose LOCAL product is the
    whole product), each with the fastest of plain_candidates() on that
    matrix, launched one after another.  Returns (parts, run(y), variants)."""
    import torch
    from paper_2203_02530_gb300 import benchmark, spmv
    parts, chosen = [], []
    y_tmp = torch.empty(offs[-1], dtype=torch.float64, device=x_d.device)
    for m, (n, rp, ci, va) in enumerate(mats):
        part = spmv.Part(n, rp, ci, va, 1)
        xm, ym = x_d[offs[m]:offs[m] + n], y_tmp[offs[m]:offs[m] + n]
        best = None
        for v, p in plain_candidates():
            try:
                part.set_op_variant(spmv.OP_LOCAL, v, p)
            except spmv.SpmvError as e:
                if e.code != spmv.EINVAL:
                    raise
                continue
            t = benchmark.time_loop(lambda: spmv.spmv_local(part.h, -1, xm, ym, s), s, reps, warmup=2)
            if best is None or t < best[0]:
                best = (t, v, p)
        part.set_op_variant(spmv.OP_LOCAL, best[1], best[2])
        parts.append(part)
        chosen.append((best[1], best[2]))

    def run(y_d):
        for m, part in enumerate(parts):
            n = mats[m][0]
            spmv.spmv_local(part.h, -1, x_d[offs[m]:offs[m] + n], y_d[offs[m]:offs[m] + n], s)
    return parts, run, chosen


def run_batched(args, world, rank, local):
    """256 independent SpMVs (n log-uniform in [1e3, 1e6]; 5-point, 7-point
    and Zipf-row matrices) in one persistent launch, against the plain form
    (each matrix through the library's tuned single-matrix product, the 256
    launches captured in one CUDA graph)."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = dist_once(world)
    from paper_2203_02530_gb300 import autotune, benchmark, spmv
    from paper_2203_02530_gb300 import workloads as W
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    mix = W.batch_mix(256, seed=5)
    mats = [m for _, m in mix]
    b = spmv.Batch(mats)
    offs = b.offsets()
    total = offs[-1]
    x = W.uniform_x(total, seed=6)
    x_d = torch.from_numpy(x).to(dev)
    y_b = torch.empty(total, dtype=torch.float64, device=dev)
    y_s = torch.empty(total, dtype=torch.float64, device=dev)
    y_p = torch.empty(total, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(device=dev)
    mrl = [(int(m[1][-1]) / m[0]) if m[0] else 0.0 for m in mats]
    tune_log = []
    lanes = autotune.tune_batch(b, x_d, y_b, s, mean_row_lengths=mrl, log=tune_log)
    batch_bytes_tuned = b.query(spmv.BQ_DEVICE_BYTES)
    if all(l == spmv.BATCH_SLICED for l in lanes):   # no product reads the CSR copy any more
        spmv.spmv_batch_release_csr(b.h)
    batch_bytes_timed = b.query(spmv.BQ_DEVICE_BYTES)
    alg = b.query(spmv.BQ_ALG_BYTES)
    batched = lambda: spmv.spmv_batch_run(b.h, x_d, y_b, s)
    separate = lambda: spmv.spmv_batch_run_separate(b.h, -1, x_d, y_s, s)
    batched()
    separate()
    s.synchronize()
    identical = bool(torch.equal(y_b, y_s))
    sampler = ClockSampler(uuid=str(getattr(props, "uuid", "")) or None)
    sampler.start()   # before the warm-up: the timed launches follow the warm-up ones directly
    for _ in range(args.warmup):
        batched()
    s.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.nvtx.range_push("timed_region")
    t_b = benchmark.time_loop(batched, s, args.steps, warmup=0)
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    t_b = max_over_ranks(dist, t_b, dev)
    per_sample = per_sample_latency(batched, s, max(args.latency_samples, args.steps))
    meas = benchmark.measurements(batched, s, max(3, args.measurements // 4))
    # the plain form: every matrix through the tuned single-matrix product
    t0 = time.perf_counter()
    parts, plain_run, chosen = plain_per_matrix(mats, offs, x_d, s)
    t_plain_tune = time.perf_counter() - t0
    plain_run(y_p)
    s.synchronize()
    d = (y_p - y_b).abs().max().item()
    rel_plain = d / max(y_b.abs().max().item(), 1e-300)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plain_run(y_p)

    def replay():
        with torch.cuda.stream(s):
            g.replay()
    t_plain_graph = benchmark.time_loop(replay, s, max(5, args.steps), warmup=args.warmup)
    t_plain_eager = benchmark.time_loop(lambda: plain_run(y_p), s, max(3, args.steps // 4), warmup=2)
    plain_sample = per_sample_latency(replay, s, max(20, args.steps))
    del g
    for part in parts:
        part.close()
    # ablation: the batch's own work items launched once per matrix
    t_sep = benchmark.time_loop(separate, s, max(3, args.steps // 4), warmup=2)
    # end to end: x from pinned host memory, the product, y back to the host
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(total, dtype=torch.float64).pin_memory()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e(chunks):   # through the library: chunked x in, products, y out, overlapped
        spmv.spmv_batch_run_host(b.h, xh, yh, chunks, s_in, s, s_out)

    chunk_t = {}
    for c in (8, 16, 32):   # the chunk count: finer chunks shorten the pipeline's fill and drain
        e2e(c)
        t0 = time.perf_counter()
        for _ in range(3):
            e2e(c)
        chunk_t[c] = (time.perf_counter() - t0) / 3
    n_chunks = min(chunk_t, key=chunk_t.get)
    k_e2e = max(5, min(args.steps, 50))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e(n_chunks)
    t_e2e_one = (time.perf_counter() - t0) / k_e2e
    # a stream of independent batched products in one call: the next
    # product's x goes in while the last one's y comes back
    spmv.spmv_batch_run_host_many(b.h, 2, xh, 0, yh, 0, n_chunks, s_in, s, s_out)
    t0 = time.perf_counter()
    spmv.spmv_batch_run_host_many(b.h, k_e2e, xh, 0, yh, 0, n_chunks, s_in, s, s_out)
    t_e2e_many = (time.perf_counter() - t0) / k_e2e
    t_e2e = min(t_e2e_one, t_e2e_many)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        reps, t0 = 0, time.perf_counter()
        byts = 0
        while time.perf_counter() - t0 < args.cpu_seconds or reps == 0:
            for m, (n, rp, ci, va) in enumerate(mats):
                oracle.csr_spmv(n, rp, ci, va, x[offs[m]:offs[m] + n])
                byts += 12 * int(rp[-1]) + 4 * (n + 1) + 16 * n
                if time.perf_counter() - t0 >= args.cpu_seconds:
                    break
            reps += 1
        secs = time.perf_counter() - t0
        cpu = {"value": round(byts / secs / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "plain CSR products of the batch's matrices in order (%.2f passes over all 256), "
                         "single-threaded C oracle, %.1f s (nproc=%d)" % (byts / alg, secs, os.cpu_count() or 0)}
    launches = spmv.spmv_batch_query(b.h, spmv.BQ_LAUNCHES, -1)
    dev_bytes = b.query(spmv.BQ_DEVICE_BYTES)   # with the host paths' device vectors
    b.close()
    if rank != 0:
        return None
    peak, peak_kind = hbm_peak()
    value = world * alg / t_b / 1e9
    nnz = int(sum(int(m[1][-1]) for m in mats))
    kname = ("batch_sliced_persistent_kernel" if all(l == spmv.BATCH_SLICED for l in lanes)
             else "batch_persistent_kernel")
    traffic = profiled_traffic("batched", kname)
    vname = {spmv.VARIANT_SELL16: "SELL16", spmv.VARIANT_SELL: "SELL", spmv.VARIANT_VECTOR: "VECTOR",
             spmv.VARIANT_MERGE: "MERGE"}
    hist = {}
    for v, p in chosen:
        k = "%s/%d" % (vname.get(v, str(v)), p)
        hist[k] = hist.get(k, 0) + 1
    return {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_b * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "batched: 256 independent SpMVs, n log-uniform in [1e3, 1e6], "
                               "5-point / 7-point / Zipf-row (mean ~10) matrices, one persistent launch",
                   "matrices": len(mats), "total_rows": total, "nnz": nnz,
                   "lanes_histogram": {str(v): lanes.count(v) for v in sorted(set(lanes))},
                   "l2": "inputs larger than L2", "alg_bytes_per_step": alg, "batch_device_bytes": batch_bytes_timed,
                   "batch_device_bytes_before_csr_release": batch_bytes_tuned,
                   "batch_device_bytes_with_host_vectors": dev_bytes},
        "percent_hbm": round(100.0 * value / world / peak, 2),
        "plain": {"form": "each matrix through the library's single-matrix product (P=1 plan, LOCAL "
                          "variant tuned per matrix), 256 launches captured in one CUDA graph",
                  "graph_ms": round(t_plain_graph * 1e3, 4), "gbs": round(alg / t_plain_graph / 1e9, 2),
                  "eager_ms": round(t_plain_eager * 1e3, 4),
                  "p50_us": round(benchmark.percentile(plain_sample, 50) * 1e6, 2),
                  "p99_us": round(benchmark.percentile(plain_sample, 99) * 1e6, 2),
                  "variants": hist, "tune_seconds": round(t_plain_tune, 1),
                  "max_abs_diff_over_max_abs_y": rel_plain},
        "speedup_vs_plain": round(t_plain_graph / t_b, 3),
        "ablation_batch_items_per_matrix": {
            "form": "the persistent kernel's work items launched once per matrix (spmv_batch_run_separate)",
            "eager_ms": round(t_sep * 1e3, 4), "gbs": round(alg / t_sep / 1e9, 2),
            "bit_identical_to_batched": identical},
        "roofline": {"bound": "hbm", "kernel": kname,
                     "achieved": round(alg / t_b / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / t_b / 1e9 / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg, "launch_us": round(t_b * 1e6, 2)},
        "latency_us": latency_block(per_sample, meas),
        "e2e": {"value": round(alg / t_e2e / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total,
                "ms_per_step": round(t_e2e * 1e3, 4),
                "path": "%s, %d chunks" % ("spmv_batch_run_host_many" if t_e2e_many <= t_e2e_one
                                           else "spmv_batch_run_host", n_chunks),
                "paths": {"spmv_batch_run_host": {"value": round(alg / t_e2e_one / 1e9, 2),
                                                  "ms_per_step": round(t_e2e_one * 1e3, 4)},
                          "spmv_batch_run_host_many": {"value": round(alg / t_e2e_many / 1e9, 2),
                                                       "ms_per_step": round(t_e2e_many * 1e3, 4)}},
                "paths_note": "spmv_batch_run_host: one batched product per call, returning after y arrived; "
                              "spmv_batch_run_host_many: %d independent products in one call, consecutive ones "
                              "overlapped" % k_e2e,
                "chunk_sweep_ms": {str(c): round(t * 1e3, 4) for c, t in sorted(chunk_t.items())}},
        "cpu_baseline": cpu, "clocks": clocks,
        "autotune_us": {k: round(t * 1e6, 1) for k, t in tune_log},
        "gpu_launches": args.steps * launches,
    }


# ---------------------------------------------------------------- serving
def run_serving(args, world, rank, local, fp64=None):
    """Poisson arrivals of SpMV requests over 64 resident matrices, each a
    block of 1..8 right-hand sides with device-drawn inputs, served with
    continuous batching against one plain launch per request."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import workloads as W
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    mix = W.serve_mix(64, seed=6)
    mats = [m for _, m in mix]
    b = spmv.Batch(mats)
    if args.serve_layout == "sliced":
        spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        spmv.spmv_batch_release_csr(b.h)   # the sliced products read only the long rows of the CSR
    resident = b.query(spmv.BQ_DEVICE_BYTES)
    sv = spmv.Server(b, n_streams=args.serve_streams, budget_bytes=40 << 30)
    rate = args.serve_rate
    arr = W.poisson_arrivals(rate, args.serve_seconds, seed=7)
    rng = np.random.default_rng(8)
    count = arr.size
    mat = rng.integers(0, len(mats), size=count).astype(np.int32)
    wid = rng.integers(1, 9, size=count).astype(np.int32)
    sd = rng.integers(0, 2**63, size=count, dtype=np.uint64)
    nn = np.array([m[0] for m in mats], dtype=np.int64)
    zz = np.array([int(m[1][-1]) for m in mats], dtype=np.int64)
    # algorithmic bytes of a request alone: its matrix once, X and Y
    req_bytes = 12 * zz[mat] + 4 * (nn[mat] + 1) + 16 * nn[mat] * wid
    warm = min(2000, count)
    sv.run(mat[:warm], wid[:warm], sd[:warm], np.zeros(warm), spmv.SERVE_BATCHED, want_hash=False)
    sv.run(mat[:warm], wid[:warm], sd[:warm], np.zeros(warm), spmv.SERVE_PLAIN, want_hash=False)
    out = {}
    clocks = None
    for name, mode in (("served", spmv.SERVE_BATCHED), ("plain", spmv.SERVE_PLAIN)):
        sampler = ClockSampler(uuid=str(getattr(props, "uuid", "")) or None)
        sampler.start()
        lat, hs, st = sv.run(mat, wid, sd, arr, mode, want_hash=True)
        c = sampler.stop()
        clocks = clocks or c
        el = st["elapsed_ns"] * 1e-9
        out[name] = {"p50_us": round(float(np.percentile(lat, 50)) * 1e6, 2),
                     "p99_us": round(float(np.percentile(lat, 99)) * 1e6, 2),
                     "p999_us": round(float(np.percentile(lat, 99.9)) * 1e6, 2),
                     "throughput_req_s": round(count / el, 1), "gbs": round(req_bytes.sum() / el / 1e9, 2),
                     "blocks": st["blocks"], "max_inflight": st["max_inflight"],
                     "admitted_while_busy": st["admitted_while_busy"],
                     "launches": spmv.spmv_serve_launches(sv.h),
                     "peak_pool_mb": round(st["peak_pool_bytes"] / 1e6, 1), "hash": hs}
    same = bool(np.array_equal(out["served"].pop("hash"), out["plain"].pop("hash")))
    # the same request mix arriving faster (near the plain form's saturation),
    # where continuous batching has queues to merge
    high = {}
    if args.serve_rate_high > 0:
        arr_h = W.poisson_arrivals(args.serve_rate_high, args.serve_seconds / 2, seed=9)
        ch = min(arr_h.size, count)
        for name, mode in (("served", spmv.SERVE_BATCHED), ("plain", spmv.SERVE_PLAIN)):
            lat, _, st = sv.run(mat[:ch], wid[:ch], sd[:ch], arr_h[:ch], mode, want_hash=False)
            el = st["elapsed_ns"] * 1e-9
            high[name] = {"p50_us": round(float(np.percentile(lat, 50)) * 1e6, 2),
                          "p99_us": round(float(np.percentile(lat, 99)) * 1e6, 2),
                          "throughput_req_s": round(ch / el, 1), "blocks": st["blocks"],
                          "launches": spmv.spmv_serve_launches(sv.h)}
        high["rate_req_s"] = args.serve_rate_high
        high["requests"] = int(ch)
    # saturation: every request present at t = 0 (the most either form can do)
    nsat = min(count, args.serve_saturation)
    sat = {}
    req_flops = 2.0 * zz[mat] * wid
    for name, mode in (("served", spmv.SERVE_BATCHED), ("plain", spmv.SERVE_PLAIN)):
        lat, _, st = sv.run(mat[:nsat], wid[:nsat], sd[:nsat], np.zeros(nsat), mode, want_hash=False)
        el = st["elapsed_ns"] * 1e-9
        if name == "served":
            sat_flops = req_flops[:nsat].sum() / el
        sat[name] = {"throughput_req_s": round(nsat / el, 1),
                     "gbs": round(req_bytes[:nsat].sum() / el / 1e9, 2), "blocks": st["blocks"],
                     "launches": spmv.spmv_serve_launches(sv.h)}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        t0, done = time.perf_counter(), 0
        byts = 0
        while time.perf_counter() - t0 < args.cpu_seconds and done < count:
            m, k = int(mat[done]), int(wid[done])
            n, rp, ci, va = mats[m]
            X = W.request_x(int(sd[done]), n, k)
            for j in range(k):
                oracle.csr_spmv(n, rp, ci, va, X[:, j])
            byts += int(req_bytes[done])
            done += 1
        secs = time.perf_counter() - t0
        cpu = {"value": round(byts / secs / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "%d requests (each column a plain CSR product), single-threaded C oracle, "
                         "%.1f s (nproc=%d)" % (done, secs, os.cpu_count() or 0)}
    sv.close()
    total = int(sum(zz) * 12 + sum(nn) * 4)
    b.close()
    peak, peak_kind = hbm_peak()
    if fp64 is None:
        fp64 = fp64_probe(dev, props)
    fpeak = 2.0 * fp64["dfma_per_s"]   # flop/s
    value = sat["served"]["gbs"]
    return {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": nsat, "warmup": warm, "ms_per_step": round(1e3 / sat["served"]["throughput_req_s"], 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals (%g req/s for %g s, %d requests) over 64 resident "
                               "matrices (7-point stencils and power-law rows, %.2f GB), width 1..8, "
                               "budget 40 GB, %d stream slots, %s layout" % (
                                   rate, args.serve_seconds, count, total / 1e9, args.serve_streams,
                                   args.serve_layout),
                   "value": "saturation throughput of the served form (all requests present at t=0; a "
                            "step is one request), per-request algorithmic bytes",
                   "resident_device_bytes": resident},
        "open_loop": out, "open_loop_high": high, "saturation": sat,
        "served_vs_plain_saturation": round(sat["served"]["gbs"] / sat["plain"]["gbs"], 3),
        "served_vs_plain_note": "the served runtime groups requests only when more blocks wait than there are "
                                "free stream slots; at %d req/s at most %d requests were in flight against %d "
                                "slots, so it issued every request alone, through the same launches as the plain "
                                "form, and the two latencies coincide; the forms differ where requests queue: "
                                "open_loop_high and saturation" % (int(args.serve_rate),
                                                                  out["served"]["max_inflight"],
                                                                  args.serve_streams),
        "results_identical_served_vs_plain": same,
        "latency_us": {"p50": out["served"]["p50_us"], "p99": out["served"]["p99_us"],
                       "plain_p50": out["plain"]["p50_us"], "plain_p99": out["plain"]["p99_us"],
                       "protocol": "arrival to observed completion, open loop, %d requests" % count},
        "roofline": {"bound": "alu",
                     "kernel": "spmm_group_kernel" if args.serve_layout == "sliced" else "spmm_kernel",
                     "achieved": round(sat_flops / 1e12, 4), "peak": round(fpeak / 1e12, 4),
                     "unit": "TFLOP/s", "frac": round(sat_flops / fpeak, 4), "traffic": None,
                     "peak_kind": "FP64 FMA pipe measured by spmv_probe_dfma in this run (2 flops per DFMA)",
                     "note": "2 flops per entry per right-hand side, over the saturation run's elapsed time "
                             "(all launches and the gaps between them)"},
        "hbm_fraction": {"achieved": sat["served"]["gbs"], "peak": peak, "unit": "GB/s",
                         "frac": round(sat["served"]["gbs"] / peak, 4),
                         "peak_kind": peak_kind, "note": "per-request algorithmic bytes at saturation"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 16, "d2h_bytes_per_step": 8,
                "note": "the saturation run is already end to end: host-timed through spmv_serve_run, the "
                        "public entry point, which takes each request's descriptor (matrix, width, seed) "
                        "from the host and returns an 8-byte hash of its Y; X is drawn on the device"},
        "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": out["served"]["launches"],
    }


# ---------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    """The CPU oracle, as it stands, on the host cores; rank 0 only."""
    if rank != 0:
        return None
    import numpy as np
    import oracle
    # calibrate: size a 150 x 150 x Z slab of the same stencil so that
    # warmup + steps samples end within the time budget
    from paper_2203_02530_gb300 import workloads as W
    budget = args.reference_budget
    n8, rp8, ci8, va8 = W.stencil_27pt(0, seed=1, dims=(8, 150, 150))
    rate, _, _, _ = oracle_rate(n8, rp8, ci8, va8, W.uniform_x(n8, seed=2), 4, 1.0)
    per_step = budget / float(args.steps + args.warmup)
    bytes_per_plane = 12 * 27 * 150 * 150
    z = int(max(4, min(150, per_step * rate * 1e9 / bytes_per_plane)))
    n, rp, ci, va = W.stencil_27pt(0, seed=1, dims=(z, 150, 150))
    x = W.uniform_x(n, seed=2)
    sample = ("27-point stencil %dx150x150 (n=%d, the full workload when z=150), P=4"
              % (z, n))
    P = 4
    pl = oracle.OraclePlan(n, rp, ci, va, P)
    nnz = int(rp[-1])
    nnz_r = sum(len(pl.export(oracle.R_COL, p)) for p in range(P))
    nsend = len(pl.export(oracle.SEND_IDX))
    rr = sum(int((np.diff(pl.export(oracle.R_PTR, p)) > 0).sum()) for p in range(P))
    alg = cpu_alg_bytes(n, nnz - nnz_r, nnz_r, rr, nsend)
    for _ in range(args.warmup):
        pl.spmv(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pl.spmv(x)
    t = time.perf_counter() - t0
    value = alg * args.steps / t / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "kind": "oracle", "cores": 1,
                         "sample": sample + ", single-threaded C oracle (nproc=%d)" % (os.cpu_count() or 0)},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


SUB_DROP = ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data")


def sub_line(line):
    """A workload's line as a sub-object of the headline line."""
    return {k: v for k, v in line.items() if k not in SUB_DROP}


def run_subs(args, world, rank, local, fp64):
    """Configs 3-5 of the metric, each measured and reported as a
    sub-object: the power-law matrix with a bounded MCTS search, the batch of
    256 matrices against its plain per-matrix form, and serving against
    plain per-request launches."""
    import copy
    out = {}
    for name in args.subs.split(","):
        a = copy.copy(args)
        a.cpu_seconds = args.sub_cpu_seconds
        a.records = None
        a.random_baseline = 0
        a.measurements = args.sub_measurements
        t0 = time.perf_counter()
        if name == "powerlaw":
            a.workload = "powerlaw"
            a.mcts_iters = args.sub_mcts_iters
            line = run_ours(a, world, rank, local, fp64=fp64)
        elif name == "batched":
            line = run_batched(a, world, rank, local)
        elif name == "serving":
            a.serve_seconds = args.sub_serve_seconds
            line = run_serving(a, world, rank, local, fp64=fp64)
        else:
            raise SystemExit("unknown sub-workload %r" % name)
        if line is not None:
            sub = sub_line(line)
            sub["wall_seconds"] = round(time.perf_counter() - t0, 1)
            out[name] = sub
        import torch
        torch.cuda.empty_cache()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--measurements", type=int, default=200,
                    help="0.01 s measurements of the best schedule (Sec. III-C.3) for its percentiles")
    ap.add_argument("--latency-samples", type=int, default=2000,
                    help="back-to-back samples timed one by one for the per-sample percentiles")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--reference-budget", type=float, default=90.0,
                    help="seconds of oracle work the reference arm aims for")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "serving"],
                    default="stencil27",
                    help="stencil27 (default): 27-point 150^3; laplacian: 5-point 64x64; "
                         "powerlaw: n=4M with MCTS over the per-rank DAG")
    ap.add_argument("--subs", default="powerlaw,batched,serving",
                    help="with the default workload on one GPU: the other configs of the metric "
                         "measured after it and reported as sub-objects ('' for none)")
    ap.add_argument("--sub-mcts-iters", type=int, default=2000,
                    help="MCTS samples of the power-law sub-object, over all orderings searched")
    ap.add_argument("--sub-serve-seconds", type=float, default=3.0)
    ap.add_argument("--sub-cpu-seconds", type=float, default=6.0)
    ap.add_argument("--sub-measurements", type=int, default=50)
    ap.add_argument("--mcts-iters", type=int, default=2000,
                    help="MCTS samples of an MCTS workload, split over the orderings searched")
    ap.add_argument("--run-modes", default="strict,relaxed,relaxed+defer",
                    help="orderings searched: strict (the kernels of a stream run in order, the paper's "
                         "semantics), relaxed (DAG-only ordering, SPMV_RUN_RELAXED), defer (remote "
                         "products sum their rows before waiting, SPMV_RUN_DEFER) and/or relaxed+defer; "
                         "the fastest is timed")
    ap.add_argument("--random-baseline", type=int, default=0,
                    help="also measure this many random programs (uniform over programs, and by "
                         "random decisions) as the search baseline")
    ap.add_argument("--records", default=None, help="JSONL log of every measured schedule")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-streams", type=int, default=32)
    ap.add_argument("--serve-rate-high", type=float, default=40000.0,
                    help="a second open-loop arrival rate, near the plain form's saturation (0: none)")
    ap.add_argument("--serve-saturation", type=int, default=20000)
    ap.add_argument("--serve-layout", choices=["sliced", "buckets"], default="sliced")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world, rank, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        import __graft_entry__
        __graft_entry__.build()
        import torch
        torch.cuda.set_device(local)
        fp64 = fp64_probe(torch.device("cuda", local), torch.cuda.get_device_properties(local))
        fp64["gather"] = gather_probe(torch.device("cuda", local), torch.cuda.get_device_properties(local))
        if args.workload == "batched":
            line = run_batched(args, world, rank, local)
        elif args.workload == "serving":
            line = run_serving(args, world, rank, local, fp64=fp64)
        else:
            line = run_ours(args, world, rank, local, fp64=fp64)
            if args.workload == "stencil27" and args.subs and world == 1:
                subs = run_subs(args, world, rank, local, fp64)
                if line is not None:
                    line.update(subs)
        if line is not None:
            line["probes"] = {"fp64": {k: v for k, v in fp64.items() if k not in ("dfma_per_s", "gather")},
                              "gather": fp64["gather"]}
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
