"""Run single building blocks of the library on a synthetic workload, for timing and profiling.

    python -m paper_2106_00449_gb300.probe --op rpy32 --workload c3_65k --reps 5

Ops: rpy32 / rpy64 (one RPY product in FP32 / FP64), saddle32, precond, forces32 (positions
and pair forces, --force-method, --potential),
lanczos32 (one M^(1/2) W), solve32 (one FP32-mixed mobility solve), step32 (one gDC step),
fcm_apply / fcm_brownian / fcm_average (fluctuating FCM of the workload's blobs in a periodic
cube of its box side, --fcm-n grid points per side).
Prints the mean wall time per call measured with CUDA events on the library's stream.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    import numpy as np
    import torch

    import paper_2106_00449_gb300 as g
    from synthetic import workloads as WL

    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="rpy32")
    ap.add_argument("--workload", default="c3_65k")
    ap.add_argument("--bodies", type=int, default=0, help="use only the first N bodies (0 = all)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--pair-kernel", type=int, default=0, help="FP32 pair kernel: 0 autotuned, 1 ordered, 2 symmetric")
    ap.add_argument("--graph", type=int, default=1, help="step32: 1 replays the step as a CUDA graph, 0 host-driven")
    ap.add_argument("--force-method", type=int, default=0, help="pair forces: 0 choose, 1 all pairs, 2 cell list")
    ap.add_argument("--fcm-n", type=int, default=512, help="fcm_*: grid points per side of the periodic cube")
    ap.add_argument("--potential", type=int, default=0,
                    help="0 soft sphere; 1, 2 with the Gaussian wells of Sec. 6.4 (A_w = 5 kT, lambda = 0.5 a)")
    args = ap.parse_args(argv)
    wl = WL.BY_NAME[args.workload]()
    if args.bodies:
        wl = wl.first_bodies(args.bodies)
    if args.op.startswith("fcm_"):
        return _fcm(args, wl)
    ctx = g.context_from_workload(wl, precision=g.FP32_MIXED, rfd_delta=1e-3, lanczos_max_iter=128,
                                  pair_kernel=args.pair_kernel, graph=args.graph, force_method=args.force_method,
                                  potential=args.potential, well_A=5.0 if args.potential else 0.0, well_lambda=0.5)
    rng = np.random.default_rng(0)
    lam = torch.as_tensor(rng.standard_normal(3 * wl.n_blobs), device=ctx.device)
    x = torch.as_tensor(rng.standard_normal(int(ctx.saddle_off[-1])), device=ctx.device)
    ops = {
        "rpy32": lambda: ctx.rpy_apply(lam, g.FP32_MIXED),
        "rpy64": lambda: ctx.rpy_apply(lam, g.FP64),
        "rpydf": lambda: ctx.rpy_apply(lam, 2),       # double-float residual product
        "saddle32": lambda: ctx.saddle_apply(x, g.FP32_MIXED),
        "precond": lambda: ctx.precond_apply(x),
        "forces32": lambda: ctx.forces(),
        "lanczos32": lambda: ctx.brownian_slip(lam),
        "solve32": lambda: ctx.mobility_solve(torch.zeros(6 * wl.n_bodies, dtype=torch.float64, device=ctx.device), lam),
        "step32": lambda: ctx.step(1),
    }
    fn = ops[args.op]
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.reps):
        fn()
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    prof = ctx.profile_read()
    print(json.dumps({"op": args.op, "workload": wl.name, "n_blobs": wl.n_blobs, "ms_per_call": ms,
                      "pairs": wl.pair_evals_per_matvec(), "pair_kernel": prof["pair_kernel"]}))
    return 0


def _fcm(args, wl) -> int:
    """fcm_apply / fcm_brownian / fcm_average: the workload's blobs in a periodic cube of its
    box side on an N^3 grid, sigma = a/sqrt(pi), envelopes cut at 3a (Sec. 4.2, Sec. 6.1)."""
    import numpy as np
    import torch

    import paper_2106_00449_gb300 as g

    ctx = g.context_from_workload(wl, precision=g.FP32_MIXED, autotune=0)
    r = ctx.blob_positions().reshape(-1, 3).contiguous()
    n = r.shape[0]
    L = float(wl.box[0])
    a = float(wl.params["a"])
    F = g.Fcm(args.fcm_n, L, a / np.sqrt(np.pi), 3.0 * a, eta=float(wl.params["eta"]), max_blobs=n, stream=ctx.stream)
    lam = torch.as_tensor(np.random.default_rng(0).standard_normal((n, 3)), device=r.device)
    F.brownian(r, 1, 0, 0, 1.0, 0.01)
    ops = {
        "fcm_apply": lambda: F.apply(r, lam),
        "fcm_brownian": lambda: F.brownian(r, 1, 0, 1, 1.0, 0.01),
        "fcm_average": lambda: F.average(r),
    }
    fn = ops[args.op]
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = F.launches
    e0.record(ctx.stream)
    for _ in range(args.reps):
        fn()
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(json.dumps({"op": args.op, "workload": wl.name, "n_blobs": n, "grid": args.fcm_n, "L": L,
                      "ms_per_call": ms, "kernels_per_call": (F.launches - l0) / args.reps}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
