"""Design-space exploration driver: measure implementations on the GPU.

Every implementation (order + stream map) is captured once as a CUDA graph
on the plan's streams and measured with the paper's protocol (samples
repeated for 0.01 s, Sec. III-C.3).  Records are appended to a JSONL log as
they are taken, so an interrupted search resumes without re-measuring
(``Recorder``); the log is also the input of the design-rule stage
(Sec. IV).
"""
import json
import os

from . import benchmark, spmv
from .mcts import Mcts
from .schedules import Dag, enumerate_schedules


class Recorder:
    """(order, stream map) -> seconds, persisted as JSON lines."""

    def __init__(self, path=None, meta=None):
        self.path = path
        self.meta = meta or {}
        self.times = {}
        if path and os.path.exists(path):
            with open(path) as f:
                for line in f:
                    line = line.strip()
                    if not line:
                        continue
                    r = json.loads(line)
                    if "order" in r:
                        self.times[(tuple(r["order"]), tuple(r["streams"]))] = r["seconds"]

    def get(self, order, smap):
        return self.times.get((tuple(order), tuple(smap)))

    def put(self, order, smap, seconds, **extra):
        self.times[(tuple(order), tuple(smap))] = seconds
        if self.path:
            rec = {"order": list(order), "streams": list(smap), "seconds": seconds}
            rec.update(self.meta)
            rec.update(extra)
            with open(self.path, "a") as f:
                f.write(json.dumps(rec) + "\n")


def graph_evaluator(part, streams, x_dev, y_dev, recorder=None, measurements=1,
                    t_measure=benchmark.T_MEASURE, relaxed=False, defer=False):
    """evaluate(order, smap) -> seconds per sample (min over `measurements`
    measurements of graph replays); `relaxed` captures each program with
    SPMV_RUN_RELAXED (DAG-only ordering), `defer` with SPMV_RUN_DEFER
    (remote products that sum their rows before waiting)."""
    flags = spmv.RUN_CAPTURE | (spmv.RUN_RELAXED if relaxed else 0) | (spmv.RUN_DEFER if defer else 0)

    def evaluate(order, smap):
        if recorder is not None:
            t = recorder.get(order, smap)
            if t is not None:
                return t
        g = part.run(order, smap, streams, x_dev, y_dev, flags)
        try:
            sample = lambda: part.run(order, smap, streams, x_dev, y_dev, spmv.RUN_REPLAY, g)
            sample()
            t = min(benchmark.measurements(sample, streams[0], measurements, t_measure))
        finally:
            spmv.spmv_graph_destroy(part.h, g)
        if recorder is not None:
            recorder.put(order, smap, t)
        return t

    return evaluate


def exhaustive(part, streams, evaluate):
    """Measure every canonical implementation; returns [(order, smap, s)]."""
    dag = Dag(part.n_ops, part.dag())
    return [(o, m, evaluate(o, m)) for o, m in enumerate_schedules(dag, len(streams))]


def mcts(part, streams, evaluate, iterations, seed=0):
    """Monte-Carlo tree search with `iterations` rollouts (Sec. III-C)."""
    dag = Dag(part.n_ops, part.dag())
    tree = Mcts(dag, len(streams), evaluate, seed=seed)
    return tree.run(iterations), tree


def random_sampling(part, streams, evaluate, count, seed=0, mode="uniform"):
    """Baseline search (Sec. VI: random sampling against MCTS at an equal
    number of measured programs): `count` distinct programs drawn at random
    and measured.  mode "uniform" draws every program with equal probability;
    "per_decision" completes each program by uniformly random legal decisions
    from the empty prefix (the rollout of Sec. III-C without a tree, which
    favours programs whose prefixes have few completions).  Returns
    [(order, smap, seconds)]."""
    from .schedules import sample_programs
    dag = Dag(part.n_ops, part.dag())
    progs = sample_programs(dag, len(streams), count, seed=seed, mode=mode)
    return [(o, m, evaluate(o, m)) for o, m in progs]
