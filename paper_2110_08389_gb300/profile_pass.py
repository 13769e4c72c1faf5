"""Smoothing steps of one smoother on one synthetic problem, or whole solves,
as a target for profilers (ncu) and quick timing.

    python -m paper_2110_08389_gb300.profile_pass [--n 4096] [--smoother tweed]
           [--dtype f32|f64] [--steps 3] [--ratio 1000] [--dim 2|3]
           [--path auto|tiled|cluster|warp|cta]
    python -m paper_2110_08389_gb300.profile_pass --solve f32_refine|f64 [--n 4096] [--steps 2]

The steps after the first (the timed ones; every solve with --solve) run
between cudaProfilerStart and cudaProfilerStop, so that
`ncu --profile-from-start off` skips the grid setup (whose kernels include
a pass of the tiled reduce per tile list) and the untimed step.

With --solve, each step is one solve of the 2D wall-clustered problem to
||r||/||f|| <= 1e-10 from u = 0 with the benchmark's parameters (tweed V(1,1),
full weighting; FP32 cycles with FP64 refinement, or FP64).

The grid has n x n (x n with --dim 3: tweed or wireframe) intervals, tanh-stretched
toward the walls (Eq. tanh) for
every smoother but wireframe, toward the centre (Eq. tanh_inv) for wireframe,
with the given max/min spacing ratio; f ~ N(0, 1) (seed 1), u = 0.  Each step
is one relaxation (red pass, then black pass) on the finest level.  Prints
the mean milliseconds per step, timed with CUDA events after one untimed step.
"""
from __future__ import annotations

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--smoother", default="tweed")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--ratio", type=float, default=1000.0)
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--path", default="auto", help="line-solve path of the finest level (3D: tiled or warp)")
    ap.add_argument("--solve", default=None, choices=["f32_refine", "f64"])
    args = ap.parse_args()
    import torch
    from . import inputs as I, mg
    if args.solve:
        return solve_steps(args)

    kind = "centre" if args.smoother == "wireframe" else "wall"
    c = I.c_for_ratio(args.n, args.ratio, kind)
    x = I.centre_coords(args.n, c) if kind == "centre" else I.wall_coords(args.n, c)
    g = mg.Grid(x, x) if args.dim == 2 else mg.Grid(x, x, x)
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    shape = g.shape(0)
    f = torch.tensor(I.rhs_gaussian(shape[0], int(np_prod(shape[1:])), 1).reshape(shape), device="cuda").to(dt)
    u = torch.zeros(shape, dtype=dt, device="cuda")
    if args.path != "auto":
        g.set_line_path(0, args.smoother, args.dtype, args.path)
    g.smooth(u, f, args.smoother, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    e0.record()
    for _ in range(args.steps - 1):
        g.smooth(u, f, args.smoother, 1)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / max(args.steps - 1, 1)
    print(f"{args.smoother} {args.dtype} n={args.n} dim={args.dim}: {ms:.4f} ms/step over {args.steps - 1} timed steps")


def solve_steps(args):
    import torch
    from . import inputs as I, mg
    c = I.c_for_ratio(args.n, args.ratio, "wall")
    x = I.wall_coords(args.n, c)
    g = mg.Grid(x, x)
    f = torch.tensor(I.rhs_gaussian(args.n + 1, args.n + 1, 1), device="cuda")
    p = mg.default_params(smoother="tweed", nu1=1, nu2=1, precision=args.solve, tol=1e-10, inner_cycles=3,
                          max_outer=20, max_cycles=200)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for k in range(args.steps):
        u = torch.zeros_like(f)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = g.solve(u, f, p)
        e1.record()
        torch.cuda.synchronize()
        print(f"solve {k}: {args.solve} n={args.n} status {r.status} cycles {r.cycles} outer {r.outer_iters} "
              f"rel {r.rel_res:.2e} {e0.elapsed_time(e1):.3f} ms")
    torch.cuda.profiler.stop()


def np_prod(a):
    out = 1
    for v in a:
        out *= v
    return out


if __name__ == "__main__":
    main()
