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
replica: weak scaling, no data-path collective).  ``--impl reference`` times
the CPU oracle on the host cores instead.
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


def kernel_source_hash():
    """Hash of the product kernels' code (comments and blank lines left out,
    so that a comment edit does not invalidate a profile)."""
    import re
    h = hashlib.sha256()
    for f in ("kernels.cu", "merge.cu", "sell.cu"):
        with open(os.path.join(ROOT, "paper_2203_02530_gb300", "csrc", f)) as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_full_launch")


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


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
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

    # the design space: every schedule (coarse DAG), MCTS samples (per-rank
    # DAG) or the single default order
    rec = search.Recorder(args.records, meta={"workload": args.workload}) if args.records else None
    if args.records:
        with open(args.records + ".dag.json", "w") as f:
            json.dump({"n_ops": part.n_ops, "edges": part.dag(), "P": P, "streams": S,
                       "names": part.op_names()}, f)
    search_cmp = None
    # the minimum of a few 0.01 s measurements per program, so that a host
    # hiccup during one measurement does not masquerade as a slow program
    evaluate = search.graph_evaluator(part, streams, x_d, y_d, recorder=rec, measurements=3
                                      if mode == "exhaustive" else 2)
    if mode == "exhaustive":
        sched = search.exhaustive(part, streams, evaluate)
    elif mode == "mcts":
        sched, _ = search.mcts(part, streams, evaluate, args.mcts_iters, seed=0)
        if args.random_baseline:
            rand = search.random_sampling(part, streams, evaluate, args.random_baseline, seed=1)
            rt = [r[2] for r in rand]
            mt = [r[2] for r in sched[:args.random_baseline]]
            search_cmp = {"samples": len(rand),
                          "random": {"best_us": round(min(rt) * 1e6, 2), "worst_us": round(max(rt) * 1e6, 2)},
                          "mcts": {"best_us": round(min(mt) * 1e6, 2), "worst_us": round(max(mt) * 1e6, 2)}}
    else:
        order = list(range(part.n_ops))
        sched = [(order, [0] * part.n_ops, evaluate(order, [0] * part.n_ops))]
    sched = sorted(sched, key=lambda r: r[2])
    order, smap, t_best = sched[0]
    spread = sched[-1][2] / sched[0][2]
    g = part.run(order, smap, streams, x_d, y_d, spmv.RUN_CAPTURE)
    step = lambda: part.run(order, smap, streams, x_d, y_d, spmv.RUN_REPLAY, g)
    part.run(order, smap, streams, x_d, y_d, spmv.RUN_EAGER)
    launches_per_step = part.query(spmv.Q_LAST_LAUNCHES)
    alg = part.query(spmv.Q_ALG_BYTES)
    alg_local = part.query(spmv.Q_ALG_BYTES_LOCAL)
    nnz_l = part.query(spmv.Q_NNZ_LOCAL)

    def timed_region():
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(uuid=str(getattr(props, "uuid", "")) or None)
        sampler.start()
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

    # the dominant kernel (LOCAL product, coarse launch), timed alone on the
    # stream the schedule launches it on, with CUDA events
    s_local = streams[smap[spmv.OP_LOCAL]]
    t_local = benchmark.time_loop(lambda: spmv.spmv_local(part.h, -1, x_d, y_d, s_local),
                                  s_local, max(50, min(args.steps, 1000)))
    peak, peak_kind = hbm_peak()
    achieved = alg_local / t_local / 1e9
    kname = {spmv.VARIANT_TILE: "csr_tile_kernel", spmv.VARIANT_VECTOR: "csr_vector_kernel",
             spmv.VARIANT_MERGE: "merge_kernel", spmv.VARIANT_PAIRS: "csr_pair_kernel",
             spmv.VARIANT_WARP: "csr_warp_kernel", spmv.VARIANT_SELL: "csr_sell_kernel",
             spmv.VARIANT_SELL16: "csr_sell_kernel"}[variant]
    traffic = profiled_traffic("%s/%d/%d" % (kname, variant, vparam))
    if traffic is None:   # the layout's bytes, measured with another param of the variant
        traffic = profiled_traffic("%s/%d" % (kname, variant))

    # paper protocol: per-measurement latency percentiles of the best schedule
    meas = benchmark.measurements(step, streams[0], args.measurements)

    # end to end through the C ABI with host buffers
    xi, yi = spmv.spmv_part_io_buffers(part.h)
    ge = part.run(order, smap, streams, xi, yi, spmv.RUN_CAPTURE)
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
    err = part.query(spmv.Q_ERROR)

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
    sm_mhz = clocks.get("sm_mhz") or 0.0
    fp64_peak = 2.0 * props.multi_processor_count * (sm_mhz or 2070.0) * 1e6   # DFMA/s
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed / args.steps * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "n": n, "nnz": int(rp[-1]), "P": P, "streams": S,
                   "granularity": ("coarse", "per-rank", "per-segment")[gran],
                   "search": mode, "schedules_measured": len(sched),
                   "best_order": order, "best_streams": smap,
                   "variant": {"local": list(tuned["local"]), "remote": list(tuned["remote"])},
                   "l2": "inputs larger than L2" if 12 * int(rp[-1]) > 129e6
                         else "L2-resident (replay latency)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "alg_bytes_per_step": alg},
        "percent_hbm": round(100.0 * value / world / peak, 2),
        "roofline": dict({"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                          "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                          "traffic": traffic, "peak_kind": peak_kind,
                          "alg_bytes_per_launch": alg_local, "launch_us": round(t_local * 1e6, 2)},
                         **({} if traffic is None else {
                             "dram_gbs": round(traffic / t_local / 1e9, 1),
                             "dram_frac": round(traffic / t_local / 1e9 / peak, 4),
                             "note": "achieved counts the CSR algorithmic bytes; the DRAM traffic of "
                                     "the launch (ncu) is `traffic`"})),
        "fp64": {"dfma_per_s": round(nnz_l / t_local / 1e9, 1), "unit": "G DFMA/s",
                 "peak": round(fp64_peak / 1e9, 1), "frac": round(nnz_l / t_local / fp64_peak, 4),
                 "note": "2 DFMA/clk/SM at the sampled SM clock"},
        "latency_us": {"p50": round(benchmark.percentile(meas, 50) * 1e6, 2),
                       "p99": round(benchmark.percentile(meas, 99) * 1e6, 2),
                       "measurements": len(meas), "protocol": "0.01 s of samples each"},
        "schedule_spread": round(spread, 4),
        "search_vs_random": search_cmp,
        "e2e": {"value": round(alg / min(t_e2e, t_e2e_graph) / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                "ms_per_step": round(min(t_e2e, t_e2e_graph) * 1e3, 4),
                "path": "spmv_apply_host_pipelined" if t_e2e <= t_e2e_graph else "spmv_apply_host",
                "paths": {"spmv_apply_host_pipelined": {"value": round(alg / t_e2e / 1e9, 2),
                                                        "ms_per_step": round(t_e2e * 1e3, 4)},
                          "spmv_apply_host": {"value": round(alg / t_e2e_graph / 1e9, 2),
                                              "ms_per_step": round(t_e2e_graph * 1e3, 4)}}},
        "cpu_baseline": cpu,
        "clocks": clocks, "remeasured": remeasured,
        "gpu_launches": launches_per_step * args.steps,
        "device_error_word": err,
        "autotune_us": {"%s %d,%d" % ("local" if k[0] == spmv.OP_LOCAL else "remote", k[1], k[2]):
                        round(v * 1e6, 1) for k, v in tune_times.items()},
    }
    return line


# ---------------------------------------------------------------- batched
def run_batched(args, world, rank, local):
    """256 independent SpMVs (n log-uniform in [1e3, 1e6]; 5-point, 7-point
    and Zipf-row matrices) in one persistent launch, against the same
    products as 256 launches (eager and captured in a CUDA graph)."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
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
    s = torch.cuda.Stream(device=dev)
    mrl = [(int(m[1][-1]) / m[0]) if m[0] else 0.0 for m in mats]
    tune_log = []
    lanes = autotune.tune_batch(b, x_d, y_b, s, mean_row_lengths=mrl, log=tune_log)
    alg = b.query(spmv.BQ_ALG_BYTES)
    batched = lambda: spmv.spmv_batch_run(b.h, x_d, y_b, s)
    separate = lambda: spmv.spmv_batch_run_separate(b.h, -1, x_d, y_s, s)
    batched()
    separate()
    s.synchronize()
    identical = bool(torch.equal(y_b, y_s))
    # the 256 launches captured once as a graph (the fairest plain form)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        separate()
    for _ in range(args.warmup):
        batched()
    s.synchronize()
    sampler = ClockSampler(uuid=str(getattr(props, "uuid", "")) or None)
    sampler.start()
    torch.cuda.nvtx.range_push("timed_region")
    t_b = benchmark.time_loop(batched, s, args.steps, warmup=0)
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    t_b = max_over_ranks(dist, t_b, dev)
    t_sep = benchmark.time_loop(separate, s, max(3, args.steps // 10), warmup=args.warmup)
    def replay():
        with torch.cuda.stream(s):
            g.replay()
    t_graph = benchmark.time_loop(replay, s, max(3, args.steps // 4), warmup=args.warmup)
    meas = benchmark.measurements(batched, s, args.measurements)
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
    t_e2e = (time.perf_counter() - t0) / k_e2e
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < args.cpu_seconds or reps == 0:
            for m, (n, rp, ci, va) in enumerate(mats):
                oracle.csr_spmv(n, rp, ci, va, x[offs[m]:offs[m] + n])
            reps += 1
        secs = time.perf_counter() - t0
        cpu = {"value": round(alg * reps / secs / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "%d passes over all 256 matrices (plain CSR products), single-threaded C "
                         "oracle, %.1f s (nproc=%d)" % (reps, secs, os.cpu_count() or 0)}
    launches = spmv.spmv_batch_query(b.h, spmv.BQ_LAUNCHES, -1)
    b.close()
    if rank != 0:
        return None
    peak, peak_kind = hbm_peak()
    value = world * alg / t_b / 1e9
    nnz = int(sum(int(m[1][-1]) for m in mats))
    return {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_b * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "batched: 256 independent SpMVs, n log-uniform in [1e3, 1e6], "
                               "5-point / 7-point / Zipf-row (mean ~10) matrices, one persistent launch",
                   "matrices": len(mats), "total_rows": total, "nnz": nnz,
                   "lanes_histogram": {str(v): lanes.count(v) for v in sorted(set(lanes))},
                   "l2": "inputs larger than L2", "alg_bytes_per_step": alg},
        "percent_hbm": round(100.0 * value / world / peak, 2),
        "separate_launches": {"eager_gbs": round(alg / t_sep / 1e9, 2),
                              "graph_gbs": round(alg / t_graph / 1e9, 2),
                              "eager_ms": round(t_sep * 1e3, 4), "graph_ms": round(t_graph * 1e3, 4),
                              "bit_identical_to_batched": identical},
        "speedup_vs_separate_graph": round(t_graph / t_b, 3),
        "speedup_vs_separate_eager": round(t_sep / t_b, 3),
        "roofline": {"bound": "hbm",
                     "kernel": ("batch_sliced_persistent_kernel" if all(l == spmv.BATCH_SLICED for l in lanes)
                                else "batch_persistent_kernel"),
                     "achieved": round(alg / t_b / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / t_b / 1e9 / peak, 4), "traffic": None, "peak_kind": peak_kind},
        "latency_us": {"p50": round(benchmark.percentile(meas, 50) * 1e6, 2),
                       "p99": round(benchmark.percentile(meas, 99) * 1e6, 2),
                       "measurements": len(meas), "protocol": "0.01 s of samples each"},
        "e2e": {"value": round(alg / t_e2e / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total,
                "ms_per_step": round(t_e2e * 1e3, 4), "path": "spmv_batch_run_host, %d chunks" % n_chunks,
                "chunk_sweep_ms": {str(c): round(t * 1e3, 4) for c, t in sorted(chunk_t.items())}},
        "cpu_baseline": cpu, "clocks": clocks,
        "autotune_us": {k: round(t * 1e6, 1) for k, t in tune_log},
        "gpu_launches": args.steps * launches,
    }


# ---------------------------------------------------------------- serving
def run_serving(args, world, rank, local):
    """Poisson arrivals of SpMV requests over 64 resident matrices, each a
    block of 1..8 right-hand sides with device-drawn inputs, served with
    continuous batching against one plain launch per request."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_2203_02530_gb300 import spmv
    from paper_2203_02530_gb300 import workloads as W
    mix = W.serve_mix(64, seed=6)
    mats = [m for _, m in mix]
    b = spmv.Batch(mats)
    if args.serve_layout == "sliced":
        spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
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
    out = {}
    for name, mode in (("served", spmv.SERVE_BATCHED), ("plain", spmv.SERVE_PLAIN)):
        lat, hs, st = sv.run(mat, wid, sd, arr, mode, want_hash=True)
        el = st["elapsed_ns"] * 1e-9
        out[name] = {"p50_us": round(float(np.percentile(lat, 50)) * 1e6, 2),
                     "p99_us": round(float(np.percentile(lat, 99)) * 1e6, 2),
                     "throughput_req_s": round(count / el, 1), "gbs": round(req_bytes.sum() / el / 1e9, 2),
                     "blocks": st["blocks"], "max_inflight": st["max_inflight"],
                     "admitted_while_busy": st["admitted_while_busy"],
                     "peak_pool_mb": round(st["peak_pool_bytes"] / 1e6, 1), "hash": hs}
    same = bool(np.array_equal(out["served"].pop("hash"), out["plain"].pop("hash")))
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
    fp64_peak = 2.0 * torch.cuda.get_device_properties(local).multi_processor_count * 2070.0e6   # DFMA/s
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
                   "value": "saturation throughput of the served form (all requests present at t=0)"},
        "open_loop": out, "saturation": sat,
        "served_vs_plain_saturation": round(sat["served"]["gbs"] / sat["plain"]["gbs"], 3),
        "results_identical_served_vs_plain": same,
        "latency_us": {"p50": out["served"]["p50_us"], "p99": out["served"]["p99_us"],
                       "protocol": "arrival to observed completion, open loop"},
        "roofline": {"bound": "alu",
                     "kernel": "spmm_group_kernel" if args.serve_layout == "sliced" else "spmm_kernel",
                     "achieved": round(sat_flops / 1e12, 4), "peak": round(fp64_peak * 2 / 1e12, 4),
                     "unit": "TFLOP/s", "frac": round(sat_flops / (fp64_peak * 2), 4), "traffic": None,
                     "peak_kind": "FP64 FMA pipe: 2 DFMA/clk/SM x 152 SMs at the maximum SM clock",
                     "note": "2 flops per entry per right-hand side, over the saturation run's elapsed time "
                             "(all launches and the gaps between them)"},
        "hbm_fraction": {"achieved": value, "peak": peak, "unit": "GB/s", "frac": round(value / peak, 4),
                         "peak_kind": peak_kind, "note": "per-request algorithmic bytes at saturation"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8,
                "note": "inputs are drawn on the device from each request's seed; the host reads "
                        "one 8-byte hash per request"},
        "cpu_baseline": cpu, "gpu_launches": sat["served"]["launches"],
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


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--measurements", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--reference-budget", type=float, default=90.0,
                    help="seconds of oracle work the reference arm aims for")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "serving"],
                    default="stencil27",
                    help="stencil27 (default): 27-point 150^3; laplacian: 5-point 64x64; "
                         "powerlaw: n=4M with MCTS over the per-rank DAG")
    ap.add_argument("--mcts-iters", type=int, default=2000)
    ap.add_argument("--random-baseline", type=int, default=0,
                    help="also measure this many random-rollout programs (search baseline)")
    ap.add_argument("--records", default=None, help="JSONL log of every measured schedule")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-streams", type=int, default=32)
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
        if args.workload == "batched":
            line = run_batched(args, world, rank, local)
        elif args.workload == "serving":
            line = run_serving(args, world, rank, local)
        else:
            line = run_ours(args, world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
