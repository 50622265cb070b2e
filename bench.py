#!/usr/bin/env python
"""Benchmark of the gDC step on GB300: steps/s at 65,520 blobs (FP32-mixed), RPY pair-evals/s.

Workload (seeded, synthetic): 2,520 rigid bodies, a third each 42-blob icosphere shells,
15-blob rods and 21-blob L-shaped boomerangs, uniform random orientations, 10% volume
fraction in a 140a cube (65,520 blobs), unbounded overlapping RPY, soft repulsion
A = 4kT/a, b = 0.1a, dt = 0.005, GMRES tol 1e-6, Lanczos tol 1e-4, RFD delta 1e-3.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c3_65k|c4|c5]
    python bench.py --op NAME [--workload W] [--reps R] ...   (one building block, for profiling)

--workload c4: 512 independent suspensions (8-128 bodies of 12-blob icosahedra, 10-blob
rods and 42-blob icospheres, 5% volume fraction each, 772,728 blobs in all) advanced in one
batched context, against the same suspensions advanced one context (one launch sequence)
per suspension.  --workload c5: 16,384 rods of 20 blobs (327,680 blobs) at 8% volume
fraction in linear shear, dt 0.002.  The default is the 65,520-blob workload above.

--op runs one building block of the library on a workload instead of the step benchmark and
prints its mean time per call (CUDA events on the library's stream): rpy32 / rpy64 / rpydf
(one RPY product in FP32 / FP64 / double-float), saddle32, precond, forces32 (positions and
pair forces), lanczos32 (one v-breve), solve32 (one FP32-mixed mobility solve), step32 (one
gDC step, --graph 0|1), fcm_apply / fcm_brownian / fcm_average (fluctuating FCM of the
workload's blobs in a periodic cube of its box side, --fcm-n grid points per side), fma_peak
(the FP32 FMA throughput probe, packed and scalar).  This is
the command the ncu captures under profiles/ run: its kernels_before_timed_calls counts the
library's kernels (all named k_*) launched before the timed calls, so `ncu -k regex:^k_ -s`
that count starts at the first timed call.

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank advances its own
independent suspension of the same size (replicas, weak scaling, no collective on the
data path); value = total steps of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gDC steps/s at 65k blobs, FP32-mixed vs FP64, residual ≤1e-6; RPY pair-evals/s"
WORKLOAD = ("c3_65k: 2,520 rigid bodies (840 each of 42-blob icosphere, 15-blob rod, 21-blob boomerang), "
            "65,520 blobs, 10% volume fraction in a 140a cube, unbounded overlapping RPY, soft repulsion")
WORKLOAD_C4 = ("c4: 512 independent suspensions of 8-128 bodies (12-blob icosahedra, 10-blob rods, 42-blob "
               "icospheres), 5% volume fraction each, 772,728 blobs, batched in one context; a step advances "
               "every suspension once")
WORKLOAD_C5 = ("c5: 16,384 rods of 20 collinear blobs, 327,680 blobs, 8% volume fraction in a 257.9a cube, "
               "linear shear u = (y, 0, 0), dt 0.002, soft repulsion")
FLOPS_PER_PAIR = 33.0          # algorithmic flops of one far-field RPY pair (FMA = 2): d 3, r^2 5, r^-2 1, r^-3 1, A 2, B 3, d.lambda 5, s 1, sums 12
FP32_LANES_PER_SM = 128


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# the FP32 pair kernels: (source file, start of the kernel, tiling macros, ncu summary)
PAIR_KERNELS = {
    1: ("rpy.cu", "template <int P, int MINB>\n__global__ void __launch_bounds__(128, MINB) k_rpy32",
        r"#define (GDC_MV_TILE) (\S+)", "k_rpy32_c3_65k.md", "k_rpy32 (ordered FP32 RPY pair kernel)"),
    2: ("sym.cu", "template <int MINB>\n__global__ void __launch_bounds__(128, MINB) k_rpy32_sym",
        r"#define (GDC_SYM_TILE) (\S+)", "k_rpy32_sym_c3_65k.md",
        "k_rpy32_sym (symmetric FP32 RPY pair kernel)"),
}


def pair_kernel_fingerprint(kind: int = 1) -> str:
    """Hash of an FP32 pair kernel's source and its tiling constants."""
    import hashlib
    import re
    fname, head, macro_re, _, _ = PAIR_KERNELS[kind]
    src = open(os.path.join(ROOT, "paper_2106_00449_gb300", "csrc", fname)).read()
    start = src.index(head)
    end = src.index("\n}\n", start) + 3
    macros = re.findall(macro_re, src)
    if kind == 2:
        macros += re.findall(r"#define (GDC_SYM_TILE) (\S+)",
                             open(os.path.join(ROOT, "paper_2106_00449_gb300", "csrc", "common.cuh")).read())
    return hashlib.sha256((src[start:end] + repr(macros)).encode()).hexdigest()[:16]


def captured_traffic(kind: int = 1):
    """DRAM bytes per launch of an FP32 pair kernel from its committed ncu summary.

    None when the kernel's source changed since that capture (the figure would be stale).
    """
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", PAIR_KERNELS[kind][3])).read()
        h = re.search(r"kernel_source_sha256: (\w+)", text)
        b = re.search(r"dram_bytes_per_launch: (\d+)", text)
        if h and b and h.group(1) == pair_kernel_fingerprint(kind):
            return int(b.group(1))
    except (OSError, ValueError):
        pass
    return None


def replica_throughput(t_local: float, steps: int, world: int, dist=None, device="cpu"):
    """Whole-job steps/s of `world` independent replicas (one suspension per rank, no data-path
    collective): every rank ran `steps` steps in t_local seconds and the job takes as long as
    the slowest rank.  Returns (steps/s of the job, the slowest rank's time)."""
    t_max = t_local
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return world * steps / t_max, t_max


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p > 0.3 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


TWIN_RECORD = os.path.join(ROOT, "profiles", "cpu_twin_step_c3_65k.md")


def twin_record() -> dict:
    """The CPU twin's full step on the 65,520-blob workload, measured once on the GPU machine's
    host cores (oracle/twin_record.py): its RPY product count and the time it spends outside
    the products.  None when the record is missing."""
    import re
    try:
        text = open(TWIN_RECORD).read()
    except OSError:
        return None
    rec = {k: float(v) for k, v in re.findall(r"^(\w+): ([-0-9.eE+]+)\s*$", text, flags=re.M)}
    return rec if "products" in rec and "non_product_seconds" in rec else None


def twin_products(wl, n: int):
    """Seconds per full-size FP64 RPY product of the CPU twin (mean of n after one untimed),
    and the OpenMP threads it used."""
    import numpy as np

    from oracle import geometry as G, twin
    lay = G.Layout(wl.templates, wl.body_tmpl)
    r = G.blob_positions(lay, wl.Y, wl.q)
    lam = np.random.default_rng(0).standard_normal(3 * lay.n_blobs)
    twin.rpy_product(r, lam, wl.params["a"], wl.params["eta"])
    t0 = time.perf_counter()
    for _ in range(n):
        twin.rpy_product(r, lam, wl.params["a"], wl.params["eta"])
    return (time.perf_counter() - t0) / n, twin.threads()


def cpu_baseline(wl, n_products: int = 3) -> dict:
    """The oracle's matrix-free FP64 twin of the step (oracle/twin.py) on the host cores.

    The sample: n_products full-size RPY products (all 65,520 blobs, pair by pair in FP64, one
    OpenMP loop), timed; a step is that product time times the products of one full twin step
    plus the step's time outside its products, both from the twin's full-size step measured
    once (profiles/cpu_twin_step_c3_65k.md)."""
    rec = twin_record()
    t_prod, threads = twin_products(wl, n_products)
    out = {"unit": "steps/s", "cores": threads, "kind": "oracle", "product_seconds": t_prod}
    if rec is None:
        out.update(value=None, sample=f"{n_products} full-size FP64 twin products, {t_prod:.2f} s each; no full-step "
                                      f"record, so no step rate")
        return out
    t_step = t_prod * rec["products"] + max(rec["non_product_seconds"], 0.0)
    out.update(value=1.0 / t_step, step_seconds=t_step,
               sample=(f"{n_products} full-size FP64 RPY products of the matrix-free twin (65,520 blobs, "
                       f"{threads} threads), {t_prod:.2f} s each, times the {int(rec['products'])} products of one "
                       f"full twin step, plus that step's {max(rec['non_product_seconds'], 0.0):.1f} s outside its "
                       f"products (both measured once on the full step: profiles/cpu_twin_step_c3_65k.md)"))
    return out


def run_reference(args, world, rank):
    """The reference arm: the oracle's matrix-free FP64 twin of the step on the host cores,
    each step one full-size product timed and scaled by the products of a full twin step."""
    if rank != 0:
        return 0
    from synthetic import workloads as WL
    wl = WL.c3_65k(seed=0)
    rec = twin_record()
    if rec is None:
        print(json.dumps({"impl": "reference", "unavailable": "no full-step record of the CPU twin "
                                                              "(profiles/cpu_twin_step_c3_65k.md)"}), flush=True)
        return 0
    for _ in range(args.warmup):
        twin_products(wl, 1)
    steps, threads = [], 1
    for _ in range(args.steps):
        t_prod, threads = twin_products(wl, 1)
        steps.append(t_prod * rec["products"] + max(rec["non_product_seconds"], 0.0))
    total = sum(steps)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 matrix-free CPU twin of the oracle"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "kind": "oracle",
                             "sample": (f"each step: one full-size FP64 RPY product of the matrix-free twin "
                                        f"(65,520 blobs, {threads} threads) timed, times the "
                                        f"{int(rec['products'])} products of one full twin step, plus its "
                                        f"{max(rec['non_product_seconds'], 0.0):.1f} s outside the products "
                                        f"(profiles/cpu_twin_step_c3_65k.md)")},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def c4_batching(g, torch, WL, common, n_susp: int) -> dict:
    """The batching leg on a sample of the c4 workload (its first n_susp suspensions, 8-128
    bodies each): steps/s of the batched context (graph replay, 3 timed steps after 3
    warm-ups) against the same suspensions one context per suspension, stepped one after
    another."""
    wl4 = WL.c4(seed=0, n_susp=n_susp)
    ctx = g.context_from_workload(wl4, precision=g.FP32_MIXED, rfd_delta=1e-3, **common)
    for _ in range(3):
        ctx.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    ctx.step(3)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    batched = 3.0 / (e0.elapsed_time(e1) / 1000.0)
    del ctx
    torch.cuda.empty_cache()
    single = per_suspension_steps(g, torch, wl4, common, 0)
    return {"workload": f"the first {n_susp} suspensions of c4 ({wl4.n_blobs} blobs, {wl4.n_bodies} bodies)",
            "batched_steps_per_s": batched, "one_context_per_suspension_steps_per_s": single["steps_per_s"],
            "batched_speedup": batched / single["steps_per_s"], "note": single["note"]}


def boomerang_wall_leg(g, torch, WL, n_susp: int, steps: int = 20) -> dict:
    """Sec. 6.2's setting: n_susp independent suspensions of one 15-blob boomerang above a
    no-slip wall (wall repulsion 23 kT, b = 0.5a, weight 0.18 kT/a, dt = 0.1 tau_D, GMRES and
    Lanczos tolerance 1e-4), advanced together in one batched context, FP64 (as the paper's
    runs) and FP32-mixed; steps/s of the whole batch by CUDA events after 3 warm-up steps."""
    wl = WL.boomerang_wall(n_susp, 1, seed=0)
    out = {"workload": f"{n_susp} suspensions of one 15-blob boomerang above a wall ({wl.n_blobs} blobs)",
           "steps": steps}
    for name, prec, delta in (("fp64", g.FP64, 1e-6), ("fp32_mixed", g.FP32_MIXED, 1e-3)):
        ctx = g.context_from_workload(wl, precision=prec, rfd_delta=delta, seed=11)
        ctx.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        inf = ctx.step(steps)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        out[name] = {"steps_per_s": steps / (e0.elapsed_time(e1) / 1000.0),
                     "lanczos_iters": inf[-1]["lanczos_iters"], "gmres_iters": inf[-1]["solve"]["iterations"],
                     "residual_max": max(i["solve"]["residual"] for i in inf)}
        del ctx
    return out


def c5_shear_leg(g, torch, WL, common, steps: int = 1) -> dict:
    """The large FP32-mixed configuration: 16,384 rods of 20 blobs (327,680 blobs) in linear
    shear, dt 0.002, the headline's tolerances; default kernels (no autotuning, to bound the
    bench's time), one warm-up step (its graph capture), then `steps` steps by CUDA events."""
    wl = WL.c5(seed=0)
    ctx = g.context_from_workload(wl, precision=g.FP32_MIXED, rfd_delta=1e-3, autotune=0, **common)
    ctx.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    inf = ctx.step(steps)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0
    out = {"workload": WORKLOAD_C5, "n_blobs": wl.n_blobs, "steps": steps, "warmup": 1,
           "steps_per_s": steps / t, "pair_evals_per_s": sum(i["pair_evals"] for i in inf) / t,
           "lanczos_iters": [i["lanczos_iters"] for i in inf], "gmres_iters": [i["solve"]["iterations"] for i in inf],
           "residual_max": max(i["solve"]["residual"] for i in inf),
           "note": "one warm-up step only (a step takes ~10 s); default kernels, not autotuned"}
    del ctx
    return out


def per_suspension_steps(g, torch, wl, common, rank):
    """The suspensions of a batch advanced one context per suspension, one after another.

    Each suspension gets its own context (graph replay, autotuned tiling); after one
    warm-up step its next step is timed with CUDA events.  A step of the whole batch is
    the sum of those times.
    """
    total, evals = 0.0, 0.0
    for s in range(wl.n_susp):
        sub = wl.subset([s])
        c = g.context_from_workload(sub, precision=g.FP32_MIXED, rfd_delta=1e-3, **common)
        c.step(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        inf = c.step(1)
        e1.record(c.stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / 1000.0
        evals += inf[0]["pair_evals"]
        del c
    return {"steps_per_s": 1.0 / total, "pair_evals_per_s": evals / total, "suspensions": wl.n_susp,
            "note": "one context per suspension, stepped one after another (one warm-up step each, then one "
                    "timed step); value = 1 / (sum of the timed steps)"}


def fcm_measure(g, torch, wl, ctx, N: int, reps: int = 3) -> dict:
    """The fluctuating-FCM operators (Sec. 4.2) on the same blobs in a periodic cube of the
    workload's box side: sigma = a/sqrt(pi), envelopes cut at 3a (Sec. 6.1), N^3 grid."""
    import numpy as np
    r = ctx.blob_positions().reshape(-1, 3).contiguous()
    n = r.shape[0]
    L, a = float(wl.box[0]), float(wl.params["a"])
    F = g.Fcm(N, L, a / np.sqrt(np.pi), 3.0 * a, eta=float(wl.params["eta"]), max_blobs=n, stream=ctx.stream)
    lam = torch.as_tensor(np.random.default_rng(0).standard_normal((n, 3)), device=r.device)
    out = {"grid": N, "L": L, "sigma": a / np.sqrt(np.pi), "R_t": 3.0 * a, "sigma_over_h": a / np.sqrt(np.pi) / (L / N),
           "n_blobs": n, "dtype": "f32 grid, f64 positions and results", "reps": reps}
    F.brownian(r, 1, 0, 0, 1.0, 0.01)
    for name, fn in (("apply_ms", lambda k: F.apply(r, lam)), ("brownian_ms", lambda k: F.brownian(r, 1, 0, k, 1.0, 0.01)),
                     ("average_ms", lambda k: F.average(r))):
        fn(0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for k in range(reps):
            fn(k + 1)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / reps
    out["grid_points_per_s_apply"] = N ** 3 / (out["apply_ms"] / 1e3)
    F.close()
    del F
    torch.cuda.empty_cache()
    # one gDC step with the FCM mobility on the same bodies in the periodic cube
    fctx = g.context_from_workload(wl, precision=g.FP64, rfd_delta=1e-3, gmres_tol=1e-4, gmres_max_iter=500,
                                   mobility=g.MOB_FCM, box_L=L, fcm_N=N, autotune=0)
    fctx.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(fctx.stream)
    inf = fctx.step(1)[0]
    e1.record(fctx.stream)
    torch.cuda.synchronize()
    out["gdc_step"] = {"steps_per_s": 1e3 / e0.elapsed_time(e1), "gmres_iters": inf["solve"]["iterations"],
                       "residual": inf["solve"]["residual"], "nu": inf["nu_min"],
                       "gmres_tol": 1e-4,
                       "note": "one timed step after one warm-up, host-driven (FCM steps are not graph-captured); "
                               "the workload's soft repulsion at minimum-image distances in the cube; GMRES to 1e-4 "
                               "as in Sec. 6.2 (the FP32 grid's rounding, a few 1e-7 of the operator, sets the floor)"}
    fctx.close()
    del fctx
    out["note"] = ("M_FCM lambda (3-D FFTs of 2 complex grids forward and back, each grid carrying two real "
                   "fields), v-breve = J L^-1 D W (stress draw, 3 complex grids forward, 2 back) and the "
                   "re-averaging J u-breve at the same positions; CUDA events on the library stream, each call "
                   "ending with a synchronisation; the grids (14 GB at 512^3) exceed L2")
    torch.cuda.empty_cache()
    return out


def fma_probe_measure(g, torch, stream, n_sm: int, iters: int = 2048, reps: int = 3):
    """FP32 FMA throughput of the library's probe kernel (8 resident 256-thread blocks per SM,
    8 independent chains per thread), packed f32x2 and scalar, CUDA events on `stream`."""
    out = torch.empty(n_sm * 8 * 256, dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    res = {"blocks": n_sm * 8, "threads_per_block": 256, "iters": iters,
           "note": "8 independent chains of FP32 pairs per thread, nothing else in the loop: "
                   "16 scalar FMAs, 8 packed f32x2 FMAs or 4 packed + 8 scalar per iteration; "
                   "pair_kernel_frac_of_packed = the pair kernel's achieved TFLOP/s / packed_tflops"}
    for mode, key in ((1, "packed_tflops"), (0, "scalar_tflops"), (2, "mixed_tflops")):
        g.fma_probe(out, mode, iters, stream)          # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = sum(g.fma_probe(out, mode, iters, stream) for _ in range(reps))
        e1.record(stream)
        torch.cuda.synchronize()
        res[key] = flops / (e0.elapsed_time(e1) / 1000.0) / 1e12
    return res


def run_op(args) -> int:
    """One building block of the library, timed with CUDA events (see --op in the module doc)."""
    import numpy as np
    import torch

    import paper_2106_00449_gb300 as g
    from synthetic import workloads as WL

    if args.op == "fma_peak":
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        r = fma_probe_measure(g, torch, torch.cuda.current_stream(), n_sm, iters=args.reps * 1024)
        print(json.dumps({"op": "fma_peak", **r}), flush=True)
        return 0
    wl = WL.BY_NAME[args.workload]()
    if args.bodies:
        wl = wl.first_bodies(args.bodies)
    if args.op.startswith("fcm_"):
        ctx = g.context_from_workload(wl, precision=g.FP32_MIXED, autotune=0)
        r = ctx.blob_positions().reshape(-1, 3).contiguous()
        n = r.shape[0]
        L, a = float(wl.box[0]), float(wl.params["a"])
        F = g.Fcm(args.fcm_n, L, a / np.sqrt(np.pi), 3.0 * a, eta=float(wl.params["eta"]), max_blobs=n,
                  stream=ctx.stream)
        lam = torch.as_tensor(np.random.default_rng(0).standard_normal((n, 3)), device=r.device)
        F.brownian(r, 1, 0, 0, 1.0, 0.01)
        ops = {"fcm_apply": lambda: F.apply(r, lam),
               "fcm_brownian": lambda: F.brownian(r, 1, 0, 1, 1.0, 0.01),
               "fcm_average": lambda: F.average(r)}
        stream, extra = ctx.stream, {"grid": args.fcm_n, "L": L}
    else:
        ctx = g.context_from_workload(wl, precision=g.FP32_MIXED, rfd_delta=1e-3, lanczos_max_iter=128,
                                      pair_kernel=args.pair_kernel, df_kernel=args.df_kernel, graph=args.graph,
                                      force_method=args.force_method, potential=args.potential,
                                      well_A=5.0 if args.potential else 0.0, well_lambda=0.5)
        rng = np.random.default_rng(0)
        n = wl.n_blobs
        lam = torch.as_tensor(rng.standard_normal(3 * n), device=ctx.device)
        x = torch.as_tensor(rng.standard_normal(int(ctx.saddle_off[-1])), device=ctx.device)
        zero_ft = torch.zeros(6 * wl.n_bodies, dtype=torch.float64, device=ctx.device)
        ops = {"rpy32": lambda: ctx.rpy_apply(lam, g.FP32_MIXED),
               "rpy64": lambda: ctx.rpy_apply(lam, g.FP64),
               "rpydf": lambda: ctx.rpy_apply(lam, 2),
               "saddle32": lambda: ctx.saddle_apply(x, g.FP32_MIXED),
               "precond": lambda: ctx.precond_apply(x),
               "forces32": lambda: ctx.forces(),
               "lanczos32": lambda: ctx.brownian_slip(lam),
               "solve32": lambda: ctx.mobility_solve(zero_ft, lam),
               "step32": lambda: ctx.step(1)}
        stream, extra = ctx.stream, {"pair_kernel": None}
    if args.op not in ops:
        raise SystemExit(f"unknown --op {args.op}; one of {sorted(ops)}")
    fn = ops[args.op]

    def launched():   # the library's own kernels launched so far (all named k_*), context and grid
        return ctx.profile_read()["launches"] + (F.launches if args.op.startswith("fcm_") else 0)

    fn()
    torch.cuda.synchronize()
    before = launched()   # kernels of the set-up and the warm-up call: what an ncu capture skips
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"op": args.op, "workload": wl.name, "n_blobs": n, "ms_per_call": e0.elapsed_time(e1) / args.reps,
           "reps": args.reps, "kernels_before_timed_calls": before,
           "kernels_per_call": (launched() - before) / args.reps, **extra}
    if "pair_kernel" in extra:
        prof = ctx.profile_read()
        out["pair_kernel"], out["df_kernel"] = prof["pair_kernel"], prof["df_kernel"]
        out["pairs"] = wl.pair_evals_per_matvec()
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="FP64 steps timed for the comparison (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-products", type=int, default=3, help="full-size twin products timed for cpu_baseline")
    ap.add_argument("--c4-suspensions", type=int, default=64,
                    help="suspensions of the c4 batching leg of the default run (0 = skip)")
    ap.add_argument("--c5-steps", type=int, default=1,
                    help="timed steps of the 327,680-blob c5 leg in the default run (0 = skip)")
    ap.add_argument("--wall-suspensions", type=int, default=36,
                    help="boomerang-above-a-wall suspensions of the default run's wall leg (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c3_65k",
                    help="c3_65k (default), c4 or c5 for the step benchmark; any synthetic workload for --op")
    ap.add_argument("--fcm-n", type=int, default=512,
                    help="grid points per side of the fluctuating-FCM measurement (0 = skip it)")
    ap.add_argument("--op", default=None, help="time one building block instead of the step (see the module doc)")
    ap.add_argument("--bodies", type=int, default=0, help="--op: only the first N bodies of the workload (0 = all)")
    ap.add_argument("--reps", type=int, default=5, help="--op: timed calls")
    ap.add_argument("--pair-kernel", type=int, default=0, help="--op: 0 autotuned, 1 ordered, 2 symmetric")
    ap.add_argument("--df-kernel", type=int, default=0,
                    help="--op: double-float kernel, 0 autotuned, 1 ordered, 3/4 symmetric at 3/4 blocks per SM")
    ap.add_argument("--graph", type=int, default=1, help="--op step32: 1 graph replay, 0 host-driven")
    ap.add_argument("--force-method", type=int, default=0, help="--op: 0 choose, 1 all pairs, 2 cell list")
    ap.add_argument("--potential", type=int, default=0, help="--op: 0 soft sphere, 1 and 2 the Sec. 6.4 wells")
    args = ap.parse_args(argv)
    if args.op:
        return run_op(args)
    if args.workload not in ("c3_65k", "c4", "c5"):
        raise SystemExit("the step benchmark runs --workload c3_65k, c4 or c5")
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    import paper_2106_00449_gb300 as g
    from synthetic import workloads as WL

    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.workload == "c4":
        wl, wl_desc = WL.c4(seed=rank), WORKLOAD_C4
    elif args.workload == "c5":
        wl, wl_desc = WL.c5(seed=rank), WORKLOAD_C5
    else:
        wl, wl_desc = WL.c3_65k(seed=rank), WORKLOAD
    common = dict(gmres_tol=1e-6, lanczos_tol=1e-4, lanczos_max_iter=128, gmres_restart=50, gmres_max_iter=500,
                  seed=1000 + rank)
    ctx = g.context_from_workload(wl, precision=g.FP32_MIXED, rfd_delta=1e-3, **common)
    stream = ctx.stream
    infos = []
    for _ in range(args.warmup):
        ctx.step(1)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=ctx.device)  # > 129 MB L2

    def timed(nsteps):
        """nsteps steps, each bracketed by CUDA events on the library's stream, L2 flushed before."""
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ts, inf = [], []
        for _ in range(nsteps):
            flush.fill_(1)                         # evict L2 between timed steps (outside the events)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf.extend(ctx.step(1))
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1000.0)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return ts, inf

    # the headline: each step replayed as one CUDA graph (the library's default)
    sampler = ClockSampler(local)
    ctx.profile(False)                         # zeroes the kernel counter; graph replay stays on
    times, infos = timed(args.steps)
    launches = ctx.profile_read()["launches"]
    clocks = sampler.stop()
    # the pair kernel's launch time: the same steps host-driven, every pair-kernel launch
    # bracketed by CUDA events (a graph's loop bodies admit no event nodes)
    ctx.profile(True)
    times_ev, infos_ev = timed(args.steps)
    prof = ctx.profile_read()
    ctx.profile(False)
    value, t_max = replica_throughput(sum(times), args.steps, world, dist, ctx.device)
    pair_evals = sum(i["pair_evals"] for i in infos)
    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    peak_tf = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    avg_s = prof["rpy32_ms"] / max(prof["rpy32_launches"], 1) / 1000.0
    achieved_tf = FLOPS_PER_PAIR * prof["pairs_per_product"] / avg_s / 1e12 if avg_s > 0 else None
    kind = int(prof.get("pair_kernel", 1)) or 1
    probe = fma_probe_measure(g, torch, stream, n_sm)
    if probe and achieved_tf:
        probe["pair_kernel_frac_of_packed"] = achieved_tf / probe["packed_tflops"]
        probe["packed_frac_of_peak"] = probe["packed_tflops"] / peak_tf
    roof_probe = {"fma_probe": probe} if probe else {}
    roof = {"bound": "alu", "kernel": PAIR_KERNELS[kind][4], "achieved": achieved_tf,
            "peak": peak_tf, "unit": "TFLOP/s", "frac": (achieved_tf / peak_tf) if achieved_tf else None,
            "traffic": captured_traffic(kind) if args.workload == "c3_65k" else None,   # captured at 65,520 blobs
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, profiles/"
                              + PAIR_KERNELS[kind][3] + " (null when the kernel source differs)",
            "peak_source": (f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {sm_max:.0f} MHz "
                            f"(sm_max_mhz of MEASURED_PEAKS.json, {peak_src})"),
            "avg_launch_ms": avg_s * 1000.0, "launches": prof["rpy32_launches"],
            "timing": "CUDA events on the library stream around every launch, over a second timed region "
                      "of the same number of steps run host-driven",
            "tiling": {"pair_kernel": "symmetric" if kind == 2 else "ordered",
                       "targets_per_thread": 4 if kind == 2 else prof["targets_per_thread"],
                       "work_waves": None if kind == 2 else prof["work_waves"],
                       "source_tiles_per_item": prof.get("sym_width") if kind == 2 else None,
                       "min_blocks_per_sm": prof.get("min_blocks_per_sm"),
                       "df_kernel": prof.get("df_kernel"),
                       "autotuned": prof["autotune_ms"] > 0},
            "flops_per_pair": FLOPS_PER_PAIR, "pairs_per_launch": prof["pairs_per_product"],
            "flop_count": ("33 flops per ordered pair (i, j), N_b^2 per launch, whichever kernel runs; the "
                           "symmetric kernel evaluates each unordered pair once for both blobs "
                           "(unique_pairs_per_launch), so it executes about 51/66 of those flops"),
            "unique_pairs_per_launch": prof.get("unique_pairs_per_product")}
    roof.update(roof_probe)
    if clocks.get("sm_mhz") and achieved_tf:
        roof["frac_at_sampled_clock"] = achieved_tf / (n_sm * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair kernels, f64 Krylov/state",
            "data": "synthetic",
            "config": {"workload": wl_desc, "n_blobs": wl.n_blobs, "n_bodies": wl.n_bodies,
                       "n_suspensions": wl.n_susp,
                       "precision": "fp32-mixed", "dt": wl.params["dt"], "gmres_tol": 1e-6, "lanczos_tol": 1e-4,
                       "rfd_delta": 1e-3, "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "pair_evals_per_s": world * pair_evals / t_max,
            "residual_max": max(i["solve"]["residual"] for i in infos),
            "lanczos_iters": [i["lanczos_iters"] for i in infos],
            "gmres_iters": [i["solve"]["iterations"] for i in infos],
            "fp64_products_per_step": statistics.mean(i["solve"]["matvecs_fp64"] for i in infos),
            "nu_range": [min(i["nu_min"] for i in infos), max(i["nu_max"] for i in infos)],
            "roofline": roof,
            "gpu_launches": int(launches),
            "host_driven": {"steps_per_s": args.steps / sum(times_ev), "steps": args.steps,
                            "note": "the same steps with host-driven Krylov loops and CUDA events around "
                                    "every pair-kernel launch; the roofline's launch time comes from here"},
            "clocks": clocks}

    if args.workload == "c4":
        line["one_suspension_per_launch"] = per_suspension_steps(g, torch, wl, common, rank)
        line["one_suspension_per_launch"]["batched_speedup"] = (
            value / world / line["one_suspension_per_launch"]["steps_per_s"])
    elif rank == 0 and world == 1 and args.c4_suspensions > 0:
        line["c4_batching"] = c4_batching(g, torch, WL, common, args.c4_suspensions)
    if args.workload == "c3_65k" and rank == 0 and world == 1 and args.wall_suspensions > 0:
        line["boomerang_wall"] = boomerang_wall_leg(g, torch, WL, args.wall_suspensions)
    if args.workload == "c3_65k" and rank == 0 and world == 1 and args.c5_steps > 0:
        line["c5_shear"] = c5_shear_leg(g, torch, WL, common, args.c5_steps)
    if args.workload != "c3_65k":
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return 0

    # end to end through the C ABI: host state in, step, host state out
    hY = torch.empty((wl.n_bodies, 3), dtype=torch.float64).pin_memory()
    hq = torch.empty((wl.n_bodies, 4), dtype=torch.float64).pin_memory()
    step0 = ctx.get_state_host_ptr(hY.data_ptr(), hq.data_ptr())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.set_state_host_ptr(hY.data_ptr(), hq.data_ptr(), step0)
        ctx.step(1, info=False)
        step0 = ctx.get_state_host_ptr(hY.data_ptr(), hq.data_ptr())
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    nbytes = 7 * 8 * wl.n_bodies
    line["e2e"] = {"value": args.e2e_steps / t_e2e, "unit": "steps/s", "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps}

    # the fluctuating-FCM operators on the same blobs (a second way to apply M, Sec. 4.2)
    if rank == 0 and world == 1 and args.fcm_n and args.workload == "c3_65k":
        line["fcm"] = fcm_measure(g, torch, wl, ctx, args.fcm_n)

    # the plain FP64 path on the same workload
    if args.fp64_steps > 0:
        del ctx
        torch.cuda.empty_cache()
        ctx64 = g.context_from_workload(wl, precision=g.FP64, rfd_delta=1e-6, **common)
        ctx64.step(1)          # warm-up: the graph capture of the FP64 step
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx64.stream)
        inf64 = ctx64.step(args.fp64_steps)
        e1.record(ctx64.stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1000.0
        line["fp64"] = {"steps_per_s": args.fp64_steps / t64, "steps": args.fp64_steps, "warmup": 1,
                        "residual_max": max(i["solve"]["residual"] for i in inf64),
                        "lanczos_iters": [i["lanczos_iters"] for i in inf64],
                        "gmres_iters": [i["solve"]["iterations"] for i in inf64],
                        "fp32_mixed_speedup": value / world / (args.fp64_steps / t64)}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(wl, n_products=args.cpu_products)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
