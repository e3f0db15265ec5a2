"""Kernel-variant autotuner for the CSR products.

Candidates are the variants compiled into the library: thread-per-row tile
geometries, vector-per-row widths, pairs, warp pipelines, the merge-path
kernel and the sliced layouts.  Each is timed on the plan's LOCAL and REMOTE
operations with CUDA events (one launch over all ranks for a coarse plan,
the P per-rank launches in a row otherwise); the fastest wins.  Results
are cached in a JSON file keyed by a matrix signature (size, entries, row
length statistics, ranks) and the device name, so a plan of the same shape
skips the search.
"""
import hashlib
import json
import os

import numpy as np

from . import spmv
from .benchmark import time_loop

CACHE = os.environ.get("SPMV_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "spmv_gb300_tune.json"))

SELL_PARAMS = (4, 8, 9, 104, 105, 106, 107) + tuple(2000 + p for p in (4, 8, 9, 104, 105, 106, 107))

CANDIDATES = ([(spmv.VARIANT_TILE, g) for g in range(5)]
              + [(spmv.VARIANT_VECTOR, w) for w in (2, 4, 8)]
              + [(spmv.VARIANT_PAIRS, w) for w in (1, 2, 4, 8, 102, 104)]
              + [(spmv.VARIANT_WARP, g) for g in range(5)]
              + [(spmv.VARIANT_MERGE, 0)]
              + [(spmv.VARIANT_SELL, u) for u in SELL_PARAMS]
              + [(spmv.VARIANT_SELL16, u) for u in SELL_PARAMS])


def signature(n, row_ptr, P, device_name):
    lens = np.diff(np.asarray(row_ptr))
    if lens.size == 0:
        stats = (0, 0, 0)
    else:
        stats = (int(lens.max()), round(float(lens.mean()), 1), round(float(lens.std()), 1))
    return "n=%d nnz=%d max=%d mean=%.1f std=%.1f P=%d dev=%s" % (
        n, int(row_ptr[-1] - row_ptr[0]), stats[0], stats[1], stats[2], P, device_name)


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def tune(part, x_dev, y_dev, stream, sig=None, candidates=CANDIDATES, reps=20,
         cache_path=CACHE, use_cache=True):
    """Pick the fastest variant for each of part's products (LOCAL, then
    REMOTE) and apply them.  Returns {"local": (variant, param),
    "remote": (variant, param), "times": {(op, variant, param): seconds}}."""
    # a plan whose DAG has one LOCAL and one REMOTE op per rank launches them
    # rank by rank, and a kernel's tail weighs more in P small launches than
    # in one: time the P per-rank launches there
    per_rank = getattr(part, "granularity", spmv.COARSE) != spmv.COARSE
    if sig:   # a cached choice holds only for the same candidate set and granularity
        sig = "%s%s cands=%s" % (sig, " per-rank" if per_rank else "",
                                 hashlib.sha256(repr(list(candidates)).encode()).hexdigest()[:12])
    cache = _load_cache(cache_path) if (use_cache and sig) else {}
    if sig and sig in cache and "local" in cache[sig]:
        e = cache[sig]
        part.set_op_variant(spmv.OP_LOCAL, *e["local"])
        part.set_op_variant(spmv.OP_REMOTE, *e["remote"])
        return {"local": tuple(e["local"]), "remote": tuple(e["remote"]),
                "times": {tuple(int(c) for c in k.split(",")): t for k, t in e["times"].items()}}
    times = {}
    ranks = list(range(part.P)) if per_rank else [-1]

    def run_local():
        for p in ranks:
            spmv.spmv_local(part.h, p, x_dev, y_dev, stream)

    def run_remote():
        for p in ranks:
            spmv.spmv_remote(part.h, p, y_dev, stream)

    ops = [(spmv.OP_LOCAL, run_local), (spmv.OP_REMOTE, run_remote)]
    best = {}
    for op, run in ops:
        usable = []
        for trial in range(2):   # two interleaved passes; keep the faster
            for v, p in candidates:
                try:
                    part.set_op_variant(op, v, p)
                except spmv.SpmvError as e:
                    if e.code != spmv.EINVAL:
                        raise
                    continue     # not applicable here (the sliced layout on skewed rows)
                t = time_loop(run, stream, reps)
                times[(op, v, p)] = min(t, times.get((op, v, p), t))
                if trial == 0:
                    usable.append((v, p))
        b = min(usable, key=lambda vp: times[(op,) + vp])
        part.set_op_variant(op, *b)
        best[op] = b
    out = {"local": best[spmv.OP_LOCAL], "remote": best[spmv.OP_REMOTE], "times": times}
    if sig and use_cache:
        cache[sig] = {"local": list(out["local"]), "remote": list(out["remote"]),
                      "times": {"%d,%d,%d" % k: t for k, t in times.items()}}
        _save_cache(cache_path, cache)
    return out


def tune_batch(batch, x_dev, y_dev, stream, mean_row_lengths=None, lanes=(0, 1, 2, 4, 8, 16, 64),
               reps=5, log=None):
    """Lanes per row for the matrices of a batch, timed on the persistent
    launch itself (one launch per matrix would be dominated by launch
    latency for small matrices): first one value for every matrix, then one
    value per class of mean row length (< 4, < 8, < 16, < 32, >= 32), each
    class tried with the others fixed.  Returns the list chosen; `log`, if
    given, receives (description, seconds) for every timing."""
    run = lambda: spmv.spmv_batch_run(batch.h, x_dev, y_dev, stream)
    best_v, best_t = None, None
    for v in lanes:
        spmv.spmv_batch_set_lanes(batch.h, -1, v)
        t = time_loop(run, stream, reps, warmup=2)
        if log is not None:
            log.append(("all %d" % v, t))
        if best_t is None or t < best_t:
            best_v, best_t = v, t
    chosen = [best_v] * batch.count
    spmv.spmv_batch_set_lanes(batch.h, -1, best_v)
    if mean_row_lengths is not None:
        edges = [4, 8, 16, 32]
        cls = [sum(mrl >= e for e in edges) for mrl in mean_row_lengths]
        for c in sorted(set(cls)):
            members = [m for m in range(batch.count) if cls[m] == c]
            cur_v, cur_t = chosen[members[0]], best_t
            for v in lanes:
                if v == cur_v:
                    continue
                for m in members:
                    spmv.spmv_batch_set_lanes(batch.h, m, v)
                t = time_loop(run, stream, reps, warmup=2)
                if log is not None:
                    log.append(("class %d -> %d" % (c, v), t))
                if t < cur_t:
                    cur_v, cur_t = v, t
                for m in members:
                    spmv.spmv_batch_set_lanes(batch.h, m, cur_v)
            for m in members:
                chosen[m] = cur_v
            best_t = cur_t
    return chosen
