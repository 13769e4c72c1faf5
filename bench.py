#!/usr/bin/env python
"""Benchmark: seconds to ||f - L u||_2 / ||f||_2 <= 1e-10 for the 4097 x 4097
tweed multigrid problem (wall-clustered tanh grid, spacing ratio 1000,
f ~ N(0,1) seed 1), FP32 smoothing + FP64 iterative refinement, with the
plain FP64 solve timed beside it, plus the roofline of the dominant kernel
(one FP32 tweed colour pass) and the CPU oracle as the baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  Multi-GPU: one independent replica per rank (the
solve does not shard); the time is the maximum over ranks.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_INTERVALS = 4096
RATIO = 1000.0
SEED = 1
TOL = 1e-10
# The timed solve of the 4097^2 workload (tests/test_gpu_fullsize.py runs exactly
# this): tweed V(1,1), full weighting, FP32 cycles (3 per refinement step)
# with the FP64 residual, update and coarsest solve of the refinement loop.
HEADLINE = dict(smoother="tweed", nu1=1, nu2=1, precision="f32_refine", tol=TOL, inner_cycles=3, max_outer=20,
                max_cycles=200, coarse_direct=0)
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "tweed_pass_f32_4097_traffic.json")
# sources whose change invalidates the stored ncu traffic of the tiled pass:
# the tiled kernels and their chunk arithmetic, their setup and layout, the launch helpers, and the tiled-path part
# of the internal header (from its "Tiled line path" comment to the Level
# struct, less the cluster pass's structs); the rest of that header (other
# paths' structs, declarations) and the checked build's part of device_util.cuh
# do not enter the tiled kernels of the timed build
TRAFFIC_SOURCES = ["tiles.cu", "tile_math.cuh", "tile_setup.cu", "tile_host.h", "device_util.cuh", "mg_internal.h#tiled"]


def traffic_key():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        fn, _, part = name.partition("#")
        text = open(os.path.join(ROOT, "paper_2110_08389_gb300", "csrc", fn), "rb").read()
        if part == "tiled":
            # the tiled path's structs, without the cluster pass's (a separate kernel)
            a = text.index(b"// Tiled line path")
            b = text.index(b"// Cluster pass", a)
            c = text.index(b"// Shapes of the line-solve kernel", b)
            text = text[a:b] + text[c:text.index(b"struct Level {", c)]
        elif fn == "device_util.cuh":
            # the checked build's part (compiled only with -DMG_CHECK)
            a = text.index(b"#ifdef MG_CHECK\n")
            text = text[:a] + text[text.index(b"#else\n", a):]
        h.update(text)
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nu", type=int, nargs=2, default=[HEADLINE["nu1"], HEADLINE["nu2"]])
    ap.add_argument("--inner", type=int, default=HEADLINE["inner_cycles"],
                    help="FP32 cycles per refinement step (each step gains at most ~1e-3 in FP32 on this grid)")
    ap.add_argument("--intervals", type=int, default=N_INTERVALS, help="intervals per side (4096: the 4097 x 4097 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--coarse-direct", type=int, default=HEADLINE["coarse_direct"], choices=[0, 1],
                    help="1: the FP32 cycles solve the finest level of at most 64x64 intervals directly, in FP32 "
                         "(default 0: every level down to the FP64 coarsest solve)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "3d"],
                    help="single: the 4097^2 solve (default); batch: 256 mixed problems solved together; "
                         "3d: the 257^3 tweed solve")
    ap.add_argument("--inner3d", type=int, default=8, help="FP32 cycles per refinement step of the 3d workload")
    ap.add_argument("--no-extras", action="store_true",
                    help="single workload: skip the smoother matrix and the batch and 3d lines added to the JSON line")
    return ap.parse_args()


def workload(n):
    from paper_2110_08389_gb300 import inputs as I
    c = I.c_for_ratio(n, RATIO, "wall")
    x = I.wall_coords(n, c)
    f = I.rhs_gaussian(n + 1, n + 1, SEED)
    return x, c, f


def config_dict(args, c):
    return {"workload": f"2D Poisson {args.intervals + 1}x{args.intervals + 1}, wall tanh c={c:.6f} (spacing ratio {RATIO:g}), "
                        f"f~N(0,1) seed {SEED}, tweed V({args.nu[0]},{args.nu[1]}), full weighting, bilinear, "
                        f"to ||r||/||f||<={TOL:g}",
            "nodes": (args.intervals + 1) ** 2, "smoother": "tweed", "nu1": args.nu[0], "nu2": args.nu[1],
            "inner_cycles": args.inner, "tol": TOL,
            "l2": f"inputs (u, f: 2 x {8 * (args.intervals + 1) ** 2 / 1e6:.0f} MB FP64) "
                  + ("larger than L2 (129 MB)" if 8 * (args.intervals + 1) ** 2 > 129e6 else "smaller than L2 (129 MB)")}


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        rows = []
        for line in open(self.out.name):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                try:
                    rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
                except ValueError:
                    pass
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[2 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        pg = dist
    return world, rank, local, pg


def max_over_ranks(v, pg, device=None):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ------------------------------------------------------------------ extras

# The comparison of 4097^2 solves: tweed and wireframe on the grids they are
# made for (wall and centre clustering, spacing ratio 1000) against
# checkerboard and alternating zebra on the same grids, and wireframe and
# alternating zebra on milder centre clustering (c = 1.5 and 2.0, where
# Sec. 6 places the limit of their convergence near c = 2.3); V(1,1) and
# V(2,2); FP64 and FP32+refine.  Caps: 100 FP64 cycles, 20 refinement steps;
# the early stop ends solves whose rate cannot reach 1e-10 under those caps.
MATRIX_GRIDS = [("wall ratio 1000", "wall", None, ("tweed", "checkerboard", "alt_zebra")),
                ("centre ratio 1000", "centre", None, ("wireframe", "checkerboard", "alt_zebra")),
                ("centre c=1.5", "centre", 1.5, ("wireframe", "alt_zebra")),
                ("centre c=2.0", "centre", 2.0, ("wireframe", "alt_zebra"))]
STATUS = {0: "ok", 4: "not converged", 5: "non-finite"}


def smoother_matrix(mg, torch, dev, n, f_h):
    """One timed solve (after an untimed one) per (grid, smoother, cycle,
    precision) of MATRIX_GRIDS; GPU time from CUDA events."""
    from paper_2110_08389_gb300 import inputs as I
    f = torch.tensor(f_h, device=dev)
    u = torch.zeros_like(f)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for label, kind, c, smoothers in MATRIX_GRIDS:
        if c is None:
            c = I.c_for_ratio(n, RATIO, kind)
        x = I.centre_coords(n, c) if kind == "centre" else I.wall_coords(n, c)
        grid = mg.Grid(x, x)
        for sm in smoothers:
            for nu in (1, 2):
                for prec in ("f64", "f32_refine"):
                    p = mg.default_params(smoother=sm, nu1=nu, nu2=nu, precision=prec, tol=TOL, max_cycles=100,
                                          max_outer=20, inner_cycles=3, early_stop=1)
                    grid.solve(u, f, p)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    r = grid.solve(u, f, p)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    out.append({"grid": label, "c": round(c, 6), "smoother": sm, "cycle": f"V({nu},{nu})",
                                "precision": prec, "status": STATUS.get(r.status, str(r.status)),
                                "s": e0.elapsed_time(e1) / 1e3, "cycles": r.cycles, "outer_iters": r.outer_iters,
                                "rel_res": r.rel_res, "conv_factor": r.conv_factor})
        grid.close()
        del grid
    return out


def workload_line(workload, args):
    """The JSON line of `bench.py --workload <workload>` (1 timed step after 1
    warm-up, no CPU baseline), run as a child process; None if it failed."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", workload, "--steps", "1", "--warmup", "1",
           "--no-cpu-baseline"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for ln in r.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)
    return {"error": f"exit {r.returncode}: {r.stderr.strip()[-300:]}"}


def host_cpu():
    """Host cores and CPU model, for the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


# ------------------------------------------------------------------ oracle

def oracle_cycles(x, f, nu, steps, warmup, threads=1):
    """Time V-cycles of the CPU oracle on the full workload from u = 0, its
    colour passes on `threads` threads (the blocks of a colour are independent;
    the result does not depend on the count).  Returns (seconds per timed
    cycle, cycles to TOL, how that count was got)."""
    import numpy as np
    import oracle
    oracle.build()
    oracle.threads(threads)
    P = oracle.Problem(x, x)
    u = np.zeros_like(f)
    fn = math.sqrt(float(np.sum(f[1:-1, 1:-1] ** 2)))
    times, rels = [], [1.0]
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        P.cycle(u, f, "tweed", nu[0], nu[1], 1, oracle.FW)
        dt = time.perf_counter() - t0
        r = P.residual(u, f)
        rels.append(math.sqrt(float(np.sum(r[1:-1, 1:-1] ** 2))) / fn)
        if k >= warmup:
            times.append(dt)
    ran = len(rels) - 1
    hit = next((k for k, v in enumerate(rels) if v <= TOL), None)
    if hit is not None:
        return statistics.mean(times), hit, f"reached 1e-10 after {hit} cycles"
    # not reached in the sample: extrapolate with the measured factor
    # (the first cycle, from u = 0, is faster than the asymptotic rate)
    rho = (rels[-1] / rels[1]) ** (1.0 / (ran - 1)) if ran >= 2 else rels[-1] / rels[0]
    more = math.ceil(math.log(TOL / rels[-1]) / math.log(rho)) if 0.0 < rho < 1.0 else float("nan")
    return statistics.mean(times), ran + more, (f"{ran} cycles run, residual {rels[-1]:.2e}; {more} more "
                                                f"extrapolated at the measured factor {rho:.4f}")


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        barrier(pg)
        return
    x, c, f = workload(args.intervals)
    t0 = time.time()
    per_cycle, cycles, how = oracle_cycles(x, f, args.nu, args.steps, args.warmup)
    value = per_cycle * cycles
    line = {"metric": "s to rel. residual 1e-10, 4097^2 tweed MG: FP32+refine vs FP64; HBM %peak",
            "value": value, "unit": "s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_cycle * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config_dict(args, c),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"one step = one FP64 V({args.nu[0]},{args.nu[1]}) cycle of the C oracle "
                                       f"(single thread) on the full grid from u = 0; value = mean s/cycle x "
                                       f"{cycles} cycles to 1e-10 ({how})"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.time() - t0}
    print(json.dumps(line), flush=True)
    barrier(pg)


# ------------------------------------------------------------------- ours

# ------------------------------------------------------------------ batch

BATCH_SIZES = (128, 256, 512, 1024)


def batch_problems(count=256, seed=2):
    """count problems: intervals per side uniform in BATCH_SIZES, spacing ratio
    log-uniform in [10, 1000], wall or centre clustering by a coin flip."""
    from paper_2110_08389_gb300 import inputs as I
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        n = int(rng.choice(BATCH_SIZES))
        ratio = float(10.0 ** rng.uniform(1.0, 3.0))
        kind = "wall" if rng.uniform() < 0.5 else "centre"
        out.append((n, ratio, kind, I.coords(n, kind, ratio=ratio)))
    return out


def run_batch(args):
    """Config 3: 256 independent 2D problems of mixed sizes and stretchings,
    FP32 cycles + FP64 refinement to 1e-10, solved as one batch
    (mg_batch_solve) and, for comparison, one after another (mg_solve)."""
    import numpy as np
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2110_08389_gb300 import build, inputs as I, mg
    build.build()
    probs = batch_problems()
    grids = [mg.Grid(x, x) for (_, _, _, x) in probs]
    fs = [torch.tensor(I.rhs_gaussian(n + 1, n + 1, 2000 + k), device="cuda") for k, (n, _, _, _) in enumerate(probs)]
    us = [torch.zeros_like(f) for f in fs]
    batch = mg.Batch(grids)
    # the paper's pairing (Sec. 6): tweed for wall clustering, wireframe for
    # clustering towards the centre
    # early_stop: a problem gives up once its last refinement step's rate
    # cannot reach the tolerance within the steps left (the centre-clustered
    # problems wireframe cannot converge, Sec. 6); the same batch without it
    # is timed once below and must converge the same problems
    def batch_params(early):
        return [mg.default_params(smoother="wireframe" if kind == "centre" else "tweed", nu1=args.nu[0],
                                  nu2=args.nu[1], precision="f32_refine", tol=TOL, inner_cycles=args.inner,
                                  max_outer=20, max_cycles=200, early_stop=early) for (_, _, kind, _) in probs]
    params = batch_params(1)
    # line-tile shapes by the autotuner: every path and warp shape of every
    # level is timed once per (level shape, smoother); later grids with the
    # same level shapes take the remembered choice
    t0 = time.perf_counter()
    for g, (_, _, kind, _) in zip(grids, probs):
        g.autotune("wireframe" if kind == "centre" else "tweed", "f32", reps=10)
    tune_s = time.perf_counter() - t0
    choices = {}
    for g, (n, _, kind, _) in zip(grids, probs):
        sm = "wireframe" if kind == "centre" else "tweed"
        choices.setdefault(f"{n + 1}^2 {sm}", [list(g.line_path(l, sm, "f32")) for l in range(g.nlev - 1)])
    for _ in range(args.warmup):
        res = batch.solve(us, fs, params)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(pg)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        l0 = mg.load().mg_kernel_launches()
        e0.record(stream)
        for _ in range(args.steps):
            res = batch.solve(us, fs, params)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = (mg.load().mg_kernel_launches() - l0) // args.steps
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, pg, torch.device("cuda", local))
    ok = sum(1 for r in res if r.status == mg.OK and r.rel_res <= TOL)
    ok_kind = {kind: sum(1 for r, p in zip(res, probs) if p[2] == kind and r.status == mg.OK)
               for kind in ("wall", "centre")}
    # the same batch without the early stop, once
    params_full = batch_params(0)
    batch.solve(us, fs, params_full)
    torch.cuda.synchronize()
    e0.record(stream)
    res_full = batch.solve(us, fs, params_full)
    e1.record(stream)
    torch.cuda.synchronize()
    full = {"s": e0.elapsed_time(e1) / 1e3,
            "converged": sum(1 for r in res_full if r.status == mg.OK and r.rel_res <= TOL),
            "same_converged_set": [r.status == mg.OK for r in res_full] == [r.status == mg.OK for r in res],
            "inner_cycles_total": sum(r.cycles for r in res_full)}
    # the same problems one after another
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(len(probs)):
        grids[k].solve(us[k], fs[k], params[k])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    # end to end: host f in, host u out
    fh = [f.cpu().pin_memory() for f in fs]
    uh = [torch.empty_like(h).pin_memory() for h in fh]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(len(probs)):
        fs[k].copy_(fh[k], non_blocking=True)
    batch.solve(us, fs, params)
    for k in range(len(probs)):
        uh[k].copy_(us[k], non_blocking=True)
    torch.cuda.synchronize()
    e2e = (time.perf_counter() - t0)
    nodes = sum((n + 1) ** 2 for (n, _, _, _) in probs)
    line = {"metric": "s to rel. residual 1e-10 for 256 mixed 2D problems, batched (FP32+refine tweed/wireframe MG)",
            "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "256 problems, n+1 in {129,257,513,1025}^2 uniform, spacing ratio log-uniform "
                                   "[10,1000], wall/centre by coin flip (seed 2), f~N(0,1), tweed (wall) / wireframe "
                                   "(centre) V(1,1), FW, to ||r||/||f||<=1e-10 or an early stop once a problem's rate cannot reach it "
                                   "within 20 refinement steps", "nodes_total": nodes, "problems": len(probs),
                       "sizes": {str(s + 1): sum(1 for p in probs if p[0] == s) for s in BATCH_SIZES}},
            "converged": ok, "converged_by_clustering": ok_kind, "early_stop": 1,
            "inner_cycles_total": sum(r.cycles for r in res), "without_early_stop": full,
            "line_paths": {"autotune_s": tune_s, "chosen": choices},
            "smoothers": "tweed (wall-clustered), wireframe (centre-clustered)",
            "problems_per_s": len(probs) / (ms / 1e3),
            "sequential_s": ms_seq / 1e3, "speedup_vs_sequential": ms_seq / ms,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 8 * nodes, "d2h_bytes_per_step": 8 * nodes},
            "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(pg)


def run_3d(args):
    """Config 5: 3D Poisson on 257^3, tanh stretching towards all six walls
    (spacing ratio 200), 3D tweed V(2,2) with full weighting (Sec. 7), to
    ||r||/||f|| <= 1e-10: FP32 cycles with FP64 refinement against FP64."""
    import numpy as np
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2110_08389_gb300 import build, inputs as I, mg
    build.build()
    n = 256
    c = I.c_for_ratio(n, 200.0)
    x = I.wall_coords(n, c)
    f_h = I.rhs_gaussian(n + 1, (n + 1) * (n + 1), 1).reshape(n + 1, n + 1, n + 1)
    grid = mg.Grid(x, x, x)
    stream = torch.cuda.current_stream()
    f = torch.tensor(f_h, device=dev)
    u = torch.zeros_like(f)
    p32 = mg.default_params(smoother="tweed", nu1=2, nu2=2, precision="f32_refine", tol=TOL,
                            inner_cycles=args.inner3d, max_outer=400, max_cycles=4000)
    p64 = mg.default_params(smoother="tweed", nu1=2, nu2=2, precision="f64", tol=TOL, max_cycles=1000)
    for _ in range(args.warmup):
        res = grid.solve(u, f, p32)
    torch.cuda.synchronize()
    barrier(pg)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = mg.kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            res = grid.solve(u, f, p32)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = (mg.kernel_launches() - l0) // max(args.steps, 1)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, pg, dev)
    u32 = u.clone()
    r64 = grid.solve(u, f, p64)
    torch.cuda.synchronize()
    e0.record(stream)
    r64 = grid.solve(u, f, p64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    err32 = float((u32 - u).abs().max() / u.abs().max())
    # end to end with host buffers
    f_pin = torch.tensor(f_h).pin_memory()
    u_pin = torch.zeros_like(f_pin).pin_memory()
    out_pin = torch.empty_like(f_pin).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u.copy_(u_pin, non_blocking=True)
    f.copy_(f_pin, non_blocking=True)
    grid.solve(u, f, p32)
    out_pin.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    e2e = time.perf_counter() - t0
    # roofline: FP32 3D tweed colour passes on the finest level, back to back
    uf = torch.zeros(f.shape, dtype=torch.float32, device=dev)
    ff = f.float()
    for k in range(4):
        grid.colour_pass(uf, ff, "tweed", k & 1)
    torch.cuda.synchronize()
    npass = 40
    e0.record(stream)
    for k in range(npass):
        grid.colour_pass(uf, ff, "tweed", k & 1)
    e1.record(stream)
    torch.cuda.synchronize()
    pass_ms = e0.elapsed_time(e1) / npass
    tiled = grid.line_path(0, "tweed", "f32")[0] == "tiled"
    nn = (n + 1) ** 3
    algo_bytes = 2 * 4 * nn
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = algo_bytes / (pass_ms * 1e-3) / 1e9
    line = {"metric": "s to rel. residual 1e-10, 257^3 3D tweed MG: FP32+refine vs FP64",
            "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"3D Poisson 257^3, wall tanh c={c:.6f} on all three axes (spacing ratio 200), "
                                   "f~N(0,1) seed 1, 3D tweed V(2,2), full weighting, trilinear, to ||r||/||f||<=1e-10",
                       "nodes": nn, "inner_cycles": args.inner3d,
                       "l2": "inputs (u, f: 2 x 136 MB FP64) larger than L2 (129 MB)"},
            "status": res.status, "rel_res": res.rel_res, "outer_iters": res.outer_iters,
            "inner_cycles_total": res.cycles, "conv_factor": res.conv_factor,
            "fp64": {"s": ms64 / 1e3, "cycles": r64.cycles, "rel_res": r64.rel_res, "status": r64.status,
                     "conv_factor": r64.conv_factor},
            "speedup_vs_fp64": ms64 / ms, "f32_refine_vs_f64_solution_maxrel": err32,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 2 * 8 * nn, "d2h_bytes_per_step": 8 * nn},
            "gpu_launches": int(launches),
            "roofline": {"kernel": "FP32 3D tweed colour pass, finest level (" +
                                   ("tile3_reduce + tile3_couple_pc + tile3_expand" if tiled else "seq3_single_kernel") + ")",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "pass_ms": pass_ms, "passes_timed": npass,
                         "launches_per_pass": 3 if tiled else 1,
                         "algo_bytes_per_pass": algo_bytes,
                         "peak_source": "hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        P = oracle.Problem3(x, x, x)
        uo = np.zeros_like(f_h)
        P.cycle(uo, f_h, 2, 2)  # untimed: builds the block partitions
        t0 = time.perf_counter()
        P.cycle(uo, f_h, 2, 2)
        per_cycle = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": per_cycle * r64.cycles, "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": f"1 FP64 V(2,2) cycle of the C 3D oracle (single thread) on the full grid "
                                          f"(after 1 untimed) = {per_cycle:.2f} s/cycle, x {r64.cycles} cycles (the "
                                          f"FP64 iteration count of this problem)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(pg)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "3d":
        return run_3d(args)
    import numpy as np
    import torch

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2110_08389_gb300 import build, mg
    build.build()
    x, c, f_h = workload(args.intervals)
    n1 = args.intervals + 1
    grid = mg.Grid(x, x)
    stream = torch.cuda.current_stream()
    f = torch.tensor(f_h, device=dev)
    u = torch.zeros((n1, n1), dtype=torch.float64, device=dev)
    p32 = mg.default_params(**dict(HEADLINE, nu1=args.nu[0], nu2=args.nu[1], inner_cycles=args.inner,
                                   coarse_direct=args.coarse_direct))
    p64 = mg.default_params(smoother="tweed", nu1=args.nu[0], nu2=args.nu[1], precision="f64", tol=TOL,
                            max_cycles=200)

    def solve(params):
        return grid.solve(u, f, params)

    for _ in range(args.warmup):
        res = solve(p32)
    torch.cuda.synchronize()
    barrier(pg)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = mg.kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            res = solve(p32)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = (mg.kernel_launches() - l0) // max(args.steps, 1)
    # the same solves again with CUDA events around every finest-level colour
    # pass, on the stream the passes are launched on (the roofline below; the
    # library launches the cycles directly while its pass timer runs)
    grid.pass_timer_begin(0, 256 * args.steps + 64)
    for _ in range(args.steps):
        solve(p32)
    torch.cuda.synchronize()
    timer = grid.pass_timer_end()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, pg, dev)
    status32 = res.status
    rel32, outer32, cyc32 = res.rel_res, res.outer_iters, res.cycles
    u32 = u.clone()

    # plain FP64 solve on the same problem (the comparison of the metric)
    solve(p64)
    torch.cuda.synchronize()
    k64 = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(k64):
        r64 = solve(p64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(e0.elapsed_time(e1) / k64, pg, dev)
    err32 = float((u32 - u).abs().max() / u.abs().max())

    # end to end through the public API with host buffers
    f_pin = torch.tensor(f_h).pin_memory()
    u_pin = torch.zeros((n1, n1), dtype=torch.float64).pin_memory()
    out_pin = torch.empty((n1, n1), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u.copy_(u_pin, non_blocking=True)
        f.copy_(f_pin, non_blocking=True)
        grid.solve(u, f, p32)
        out_pin.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, pg, dev)

    # roofline of the dominant kernel: the FP32 tweed colour pass on the finest
    # level (tile_reduce + tile_couple_pc + tile_expand), timed live in the solves
    # (each stage includes the event-record gap of about 2 us)
    npass = max(timer["passes"], 1)
    stage_ms = [v / npass for v in timer["stage_ms"]]
    pass_ms = sum(stage_ms)
    algo_bytes = 2 * 4 * n1 * n1  # read u (w) + f of the colour (w/2) + write u of the colour (w/2), w = 4 B
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = algo_bytes / (pass_ms * 1e-3) / 1e9
    traffic = None
    if os.path.exists(TRAFFIC):
        tr = json.load(open(TRAFFIC))
        if tr.get("sources_sha256") == traffic_key():
            traffic = tr.get("traffic_bytes_per_pass")

    line = {"metric": "s to rel. residual 1e-10, 4097^2 tweed MG: FP32+refine vs FP64; HBM %peak",
            "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic", "config": config_dict(args, c),
            "coarse_direct": (f"the FP32 cycles stop at level {grid.direct_level} ({grid.shape(grid.direct_level)[0]}^2) and "
                              "solve it directly (one kernel); FP64 cycles use every level"
                              if args.coarse_direct and grid.direct_level >= 0 else "off"),
            "status": status32, "rel_res": rel32, "outer_iters": outer32, "inner_cycles_total": cyc32,
            "fp64": {"s": ms64 / 1e3, "cycles": r64.cycles, "rel_res": r64.rel_res, "status": r64.status},
            "speedup_vs_fp64": ms64 / ms, "f32_refine_vs_f64_solution_maxrel": err32,
            "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": 2 * 8 * n1 * n1,
                    "d2h_bytes_per_step": 8 * n1 * n1},
            "gpu_launches": int(launches),
            "roofline": {"kernel": "FP32 tweed colour pass, finest level (tile_reduce + tile_couple_pc + tile_expand)",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "pass_ms": pass_ms,
                         "passes_timed": timer["passes"], "launches_per_pass": 3,
                         "stage_ms": {"tile_reduce": stage_ms[0], "tile_couple_pc": stage_ms[1],
                                      "tile_expand": stage_ms[2]},
                         "algo_bytes_per_pass": algo_bytes,
                         "peak_source": "hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"},
            "clocks": clk.summary()}

    if rank == 0 and world == 1 and not args.no_extras:
        # smoother comparison at full size, then the batched and 3D workloads
        # (child processes, so that their grids do not share this one's memory)
        del grid
        torch.cuda.empty_cache()
        line["smoother_matrix"] = smoother_matrix(mg, torch, dev, args.intervals, f_h)
        torch.cuda.empty_cache()
        for wl in ("batch", "3d"):
            sub = workload_line(wl, args)
            keep = ("metric", "value", "unit", "config", "status", "rel_res", "outer_iters", "inner_cycles_total",
                    "converged", "converged_by_clustering", "sequential_s", "speedup_vs_sequential", "fp64",
                    "speedup_vs_fp64", "e2e", "gpu_launches", "roofline", "problems_per_s", "error")
            line[wl] = {k: v for k, v in sub.items() if k in keep}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        per_cycle, _, _ = oracle_cycles(x, f_h, args.nu, 3, 1)
        cycles = r64.cycles
        allc = os.cpu_count() or 1
        per_cycle_all, _, _ = oracle_cycles(x, f_h, args.nu, 3, 1, threads=allc)
        threads_all = oracle.threads(0)
        line["cpu_baseline"] = {"value": per_cycle * cycles, "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": f"mean of 3 FP64 V({args.nu[0]},{args.nu[1]}) cycles of the C oracle "
                                          f"(single thread) on the full grid (after 1 untimed) = {per_cycle:.2f} "
                                          f"s/cycle, x {cycles} cycles (the FP64 iteration count of this problem)",
                                "all_cores": {"value": per_cycle_all * cycles, "unit": "s", "cores": threads_all,
                                              "s_per_cycle": per_cycle_all,
                                              "sample": "the same, the oracle's colour passes on every host core "
                                                        "(OpenMP over the independent blocks of a colour; the "
                                                        "residual and the transfers stay serial)"},
                                "host": host_cpu()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(pg)


if __name__ == "__main__":
    main()
