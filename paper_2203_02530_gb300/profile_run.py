"""Run a few launches of one product for an external profiler (ncu).

    python -m paper_2203_02530_gb300.profile_run --workload stencil27 \\
        --variant 1 2 --op local --launches 3

builds the workload's plan (27-point stencil 150^3 with P = 4, or the n = 4M
power-law matrix with P = 8 per-rank ops), selects the product variant for the
chosen operation, and launches it `--launches` times on one stream.  With
`--workload batch` it builds the batched mix of `--matrices` matrices instead,
sets every matrix to `--lanes` (64: the sliced layout) and launches
spmv_batch_run.  Nothing is timed here; pair it with
`ncu -k regex:<kernel> -s <launches-1> -c 1`.  `--workload serve` runs a burst
of `--requests` requests through the serving runtime over its 64-matrix mix in
the sliced layout.  The power-law matrix is cached
as .npz under --cache-dir so a plain run and the profiled run do not both
generate it.
"""
import argparse
import os

import numpy as np


def load(workload, cache_dir):
    from . import workloads as W
    if workload == "stencil27":
        n, rp, ci, va = W.stencil_27pt(150, seed=1)
        return n, rp, ci, va, W.uniform_x(n, seed=2), 4, 0
    path = os.path.join(cache_dir, "powerlaw_4M_seed3.npz")
    if os.path.exists(path):
        z = np.load(path)
        n, rp, ci, va = int(z["n"]), z["rp"], z["ci"], z["va"]
    else:
        n, rp, ci, va = W.powerlaw(4_000_000, seed=3)
        os.makedirs(cache_dir, exist_ok=True)
        np.savez(path, n=n, rp=rp, ci=ci, va=va)
    return n, rp, ci, va, W.uniform_x(n, seed=4), 8, 1


def run_batch(args):
    import torch
    from . import spmv
    from . import workloads as W
    mats = [m for _, m in W.batch_mix(args.matrices, seed=5)]
    b = spmv.Batch(mats)
    spmv.spmv_batch_set_lanes(b.h, -1, args.lanes)
    total = b.offsets()[-1]
    x_d = torch.from_numpy(W.uniform_x(total, seed=6)).cuda()
    y_d = torch.zeros(total, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()   # made on the current stream, used on s
    s = torch.cuda.Stream()
    for _ in range(args.launches):
        spmv.spmv_batch_run(b.h, x_d, y_d, s)
    s.synchronize()
    print("launched %d x batch of %d matrices (%d rows, %d entries), lanes %d" % (
        args.launches, args.matrices, total, b.query(spmv.BQ_TOTAL_NNZ), args.lanes))
    b.close()
    return 0


def run_serve(args):
    """The serving mix (64 matrices, sliced layout) under a burst of
    `--requests` requests (all present at t = 0), served in groups."""
    import numpy as np
    from . import spmv
    from . import workloads as W
    mats = [m for _, m in W.serve_mix(64, seed=6)]
    b = spmv.Batch(mats)
    spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
    sv = spmv.Server(b, n_streams=32, budget_bytes=40 << 30)
    rng = np.random.default_rng(8)
    cnt = args.requests
    mat = rng.integers(0, len(mats), size=cnt).astype(np.int32)
    wid = rng.integers(1, 9, size=cnt).astype(np.int32)
    sd = rng.integers(0, 2**63, size=cnt, dtype=np.uint64)
    lat, _, st = sv.run(mat, wid, sd, np.zeros(cnt), spmv.SERVE_BATCHED, want_hash=False)
    print("served %d requests in %d blocks, %d launches" % (cnt, st["blocks"], spmv.spmv_serve_launches(sv.h)))
    sv.close()
    b.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", choices=["stencil27", "powerlaw", "batch", "serve"], default="stencil27")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--matrices", type=int, default=64)
    ap.add_argument("--lanes", type=int, default=64)
    ap.add_argument("--variant", type=int, nargs=2, default=[1, 2], metavar=("VARIANT", "PARAM"))
    ap.add_argument("--op", choices=["local", "remote"], default="local")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--rank", type=int, default=-1,
                    help="launch the operation of this rank only (-1: one launch over all ranks; -2: one "
                         "launch per rank, rank after rank, as a per-rank schedule runs them)")
    ap.add_argument("--cache-dir", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build"),
                    help="where the generated power-law matrix is cached (default: the package's "
                         "ignored build folder)")
    args = ap.parse_args(argv)
    import torch
    from . import spmv
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    n, rp, ci, va, x, P, gran = load(args.workload, args.cache_dir)
    part = spmv.Part(n, rp, ci, va, P, gran)
    del ci, va
    kind = spmv.OP_LOCAL if args.op == "local" else spmv.OP_REMOTE
    part.set_op_variant(kind, *args.variant)
    x_d = torch.from_numpy(x).cuda()
    y_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()   # made on the current stream, used on another
    s = torch.cuda.Stream()
    spmv.spmv_pack(part.h, -1, x_d, s)
    spmv.spmv_halo_copy(part.h, -1, s)
    ranks = list(range(P)) if args.rank == -2 else [args.rank]
    for _ in range(args.launches):
        for r in ranks:
            if kind == spmv.OP_LOCAL:
                spmv.spmv_local(part.h, r, x_d, y_d, s)
            else:
                spmv.spmv_remote(part.h, r, y_d, s)
    s.synchronize()
    err = part.query(spmv.Q_ERROR)
    part.close()
    print("launched %d x %s of rank %d (variant %d/%d); error word %d" % (
        args.launches, args.op, args.rank, args.variant[0], args.variant[1], err))
    return 0 if err == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
