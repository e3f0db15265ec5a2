"""Multi-rank host logic of bench.py on CPU: the timing of a step is the
maximum over ranks (gloo, world size 2), as the contract for N > 1 asks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(dist, 0.25 + rank)      # rank 1 is the slow one
        w, r, l = bench.dist_env()
        out.put((rank, t, w, r))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res) == [(0, 1.25, 2, 0), (1, 1.25, 2, 1)]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.dist_init(1, "gloo") is None
