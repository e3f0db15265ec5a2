"""Run a few launches of one product for an external profiler (ncu).

    python -m paper_2203_02530_gb300.profile_run --workload stencil27 \\
        --variant 1 2 --op local --launches 3

builds the workload's plan (27-point stencil 150^3 with P = 4, or the n = 4M
power-law matrix with P = 8 per-rank ops), selects the product variant for the
chosen operation, and launches it `--launches` times on one stream.  Nothing is
timed here; pair it with `ncu -k regex:<kernel> -s <launches-1> -c 1`.  The
power-law matrix is cached as .npz under --cache-dir so a plain run and the
profiled run do not both generate it.
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
        np.savez(path, n=n, rp=rp, ci=ci, va=va)
    return n, rp, ci, va, W.uniform_x(n, seed=4), 8, 1


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", choices=["stencil27", "powerlaw"], default="stencil27")
    ap.add_argument("--variant", type=int, nargs=2, default=[1, 2], metavar=("VARIANT", "PARAM"))
    ap.add_argument("--op", choices=["local", "remote"], default="local")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--cache-dir", default="/tmp")
    args = ap.parse_args(argv)
    import torch
    from . import spmv
    n, rp, ci, va, x, P, gran = load(args.workload, args.cache_dir)
    part = spmv.Part(n, rp, ci, va, P, gran)
    del ci, va
    kind = spmv.OP_LOCAL if args.op == "local" else spmv.OP_REMOTE
    part.set_op_variant(kind, *args.variant)
    x_d = torch.from_numpy(x).cuda()
    y_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    spmv.spmv_pack(part.h, -1, x_d, s)
    spmv.spmv_halo_copy(part.h, -1, s)
    for _ in range(args.launches):
        if kind == spmv.OP_LOCAL:
            spmv.spmv_local(part.h, -1, x_d, y_d, s)
        else:
            spmv.spmv_remote(part.h, -1, y_d, s)
    s.synchronize()
    err = part.query(spmv.Q_ERROR)
    part.close()
    print("launched %d x %s (variant %d/%d); error word %d" % (args.launches, args.op,
                                                               args.variant[0], args.variant[1], err))
    return 0 if err == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
