"""One full matrix-free FP64 gDC step of the CPU twin on the 65,520-blob workload, timed.

TEST INFRASTRUCTURE ONLY.  Runs oracle/twin.py's step (FP64 pairs, Lanczos to 1e-4 on the
block-preconditioned operator, GMRES to 1e-6, RFD delta 1e-6 of Sec. 6.2) on every host
core once and prints one JSON line: the step's wall time, its RPY product count and the
time of one product measured separately, so that a bounded sample of products can later be
converted into a step rate.

    python -m oracle.twin_record [--workload c3_65k] [--seed 0] [--products-only N]

With --products-only N it times N full-size RPY products and no step (for workloads whose
step takes hours on the host, such as the 327,680-blob c5).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    import numpy as np

    from oracle import geometry as G, philox, twin
    from synthetic import workloads as WL

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c3_65k")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--products-only", type=int, default=0)
    args = ap.parse_args(argv)
    wl = WL.BY_NAME[args.workload](seed=args.seed)
    lay = G.Layout(wl.templates, wl.body_tmpl)
    p = twin.TwinParams.from_dict(dict(wl.params, rfd_delta=1e-6, lanczos_tol=1e-4, gmres_tol=1e-6))
    W = philox.normals(1000, 0, 0, 0, 3 * lay.n_blobs)
    Wt = philox.normals(1000, 0, 0, 1, 6 * lay.n_bodies)
    r = G.blob_positions(lay, wl.Y, wl.q)
    if args.products_only > 0:
        ts = []
        for _ in range(args.products_only):
            t0 = time.perf_counter()
            twin.rpy_product(r, W, p.a, p.eta)
            ts.append(time.perf_counter() - t0)
        t = sum(ts) / len(ts)
        print(json.dumps({"workload": wl.name, "n_blobs": lay.n_blobs, "threads": twin.threads(),
                          "products": len(ts), "product_seconds": t,
                          "pair_evals_per_s": float(lay.n_blobs) ** 2 / t}), flush=True)
        return 0
    t0 = time.perf_counter()
    twin.rpy_product(r, W, p.a, p.eta)
    t_prod = time.perf_counter() - t0
    out = twin.gdc_step(lay, wl.Y, wl.q, W, Wt, p)
    rec = {"workload": wl.name, "n_blobs": lay.n_blobs, "threads": twin.threads(), "step_seconds": out["seconds"],
           "products": out["products"], "product_seconds": t_prod, "k0": out["k0"], "k_mid": out["k_mid"],
           "gmres_iters": out["gmres_iters"], "gmres_cycles": out["gmres_cycles"], "residual": out["residual"],
           "nu": out["nu"], "non_product_seconds": out["seconds"] - out["products"] * t_prod}
    print(json.dumps(rec), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
