"""Empirical measurement of one implementation (Sec. III-C.3, rollout).

A *sample* is one invocation of the program; a *measurement* repeats samples
until t_measure = 0.01 s has elapsed and estimates the program's time as
t_measure / n_samples.  With P virtual ranks on one GPU the maximum over
ranks is the single GPU timeline.  Samples are graph replays (or eager
issues) timed with CUDA events on the origin stream; the number of samples
per measurement is found by doubling batches.
"""
import time

from .constants import PAPER

T_MEASURE = PAPER.t_measure   # seconds (Sec. III-C.3)


def _events(torch):
    return (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))


def measure(sample, stream, t_measure=T_MEASURE, max_samples=1 << 20):
    """One measurement: returns (seconds per sample, n_samples)."""
    import torch
    e0, e1 = _events(torch)
    n = 1
    while True:
        e0.record(stream)
        for _ in range(n):
            sample()
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        if t >= t_measure or n >= max_samples:
            return t / n, n
        # aim past t_measure on the next batch
        n = min(max_samples, max(2 * n, int(n * t_measure / max(t, 1e-7) * 1.2) + 1))


def measurements(sample, stream, count, t_measure=T_MEASURE):
    """`count` measurements; returns the list of per-sample times (s)."""
    return [measure(sample, stream, t_measure)[0] for _ in range(count)]


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    f = int(k)
    c = min(f + 1, len(v) - 1)
    return v[f] + (v[c] - v[f]) * (k - f)


def time_loop(sample, stream, reps, warmup=3):
    """Mean seconds per sample over `reps` back-to-back samples."""
    import torch
    for _ in range(warmup):
        sample()
    e0, e1 = _events(torch)
    e0.record(stream)
    for _ in range(reps):
        sample()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / reps


def wall(fn):
    t0 = time.perf_counter()
    r = fn()
    return time.perf_counter() - t0, r
