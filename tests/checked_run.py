"""Run by tests/test_gpu_checked.py in a child process whose TWEEDMG_LIB names
the checked build of the library (build.py --checked): the small-grid parity
set of the GPU path, every call of which must return MG_OK with no bad index
recorded by any kernel, on inputs poisoned with NaN where a kernel must not
read (the relaxed colour's own nodes before a colour pass; the outputs of the
transfers before they are written), and the 3D tiled tweed path on a 64^3
level.  Prints one line "checked ok <calls>" or raises."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2110_08389_gb300 import inputs as I, mg  # noqa: E402

CHECKED = 0x80000000


def own_nodes(P, smoother, colour, lev=0):
    part, owner = P.partition(smoother, lev), P.owner(smoother, lev)
    m = np.zeros(owner.shape, dtype=bool)
    inside = owner >= 0
    m[inside] = part[owner[inside], 1] == colour
    return m


def main():
    import torch
    lib = mg.load()
    assert mg.LIB_PATH == os.environ["TWEEDMG_LIB"]
    assert lib.mg_check_word() == CHECKED, "not the checked build"
    calls = 0
    rng = np.random.default_rng(17)
    grids = [(64, 64, "wall", 3.0), (96, 136, "centre", 2.0), (200, 72, "wall", 2.5), (1024, 1024, "wall", 3.0)]
    for nx, ny, kind, c in grids:
        cx = {"wall": I.wall_coords, "centre": I.centre_coords}[kind]
        x, y = cx(nx, c), cx(ny, c)
        g, P = mg.Grid(x, y), oracle.Problem(x, y)
        print(f"grid {nx}x{ny} {kind}", flush=True)
        sms = ["tweed", "zebra_x", "checkerboard"] + (["wireframe"] if nx < 1024 else [])
        for sm in sms:
            for colour in (0, 1):
                u0 = rng.standard_normal(P.shape(0))
                f = rng.standard_normal(P.shape(0))
                mine = own_nodes(P, "checkerboard" if sm == "checkerboard" else sm, colour) \
                    if sm != "checkerboard" else None
                if mine is None:
                    jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
                    mine = ((ii + jj) % 2 == colour) & (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
                u0[mine] = np.nan  # the pass must not read its own colour
                ref = P.colour_pass(np.where(mine, 0.0, u0), f, sm, colour)
                paths = ["auto"] + (["tiled", "cluster"] if nx >= 1024 and sm != "checkerboard" else [])
                for dt in ("f64", "f32"):
                    for path in paths:
                        if path == "cluster" and dt == "f64":
                            continue
                        if path != "auto":
                            g.set_line_path(0, sm, dt, path)
                        tdt = torch.float64 if dt == "f64" else torch.float32
                        ud = torch.tensor(u0, dtype=tdt, device="cuda")
                        print(f"  colour pass {sm} {colour} {dt} {path}", flush=True)
                        g.colour_pass(ud, torch.tensor(f, dtype=tdt, device="cuda"), sm, colour)
                        calls += 1
                        got = ud.double().cpu().numpy()
                        if path != "auto":
                            g.set_line_path(0, sm, dt, "auto")
                        assert np.all(np.isfinite(got[mine])), (nx, sm, colour, dt, path)
                        tol = 1e-10 if dt == "f64" else 2e-3
                        err = np.abs(got[mine] - ref[mine]).max() / max(1.0, np.abs(ref[mine]).max())
                        assert err <= tol, (nx, sm, colour, dt, path, err)
        # transfers into NaN-poisoned outputs
        u = rng.standard_normal(P.shape(0))
        f = rng.standard_normal(P.shape(0))
        for restriction in (mg.HW, mg.FW):
            ud, fd = torch.tensor(u, device="cuda"), torch.tensor(f, device="cuda")
            fc = torch.full(P.shape(1), float("nan"), dtype=torch.float64, device="cuda")
            uc = torch.full(P.shape(1), float("nan"), dtype=torch.float64, device="cuda")
            g.residual_restrict(ud, fd, fc, uc, restriction=restriction)
            calls += 1
            ref = P.restrict(P.residual(u, f), oracle.FW if restriction == mg.FW else oracle.HW)
            gfc = fc.cpu().numpy()
            assert np.all(np.isfinite(gfc[1:-1, 1:-1])) and np.all(uc.cpu().numpy()[1:-1, 1:-1] == 0.0)
            assert np.abs(gfc[1:-1, 1:-1] - ref[1:-1, 1:-1]).max() <= 1e-12 * np.abs(ref).max()
        # a short FP64 solve and an FP32+refine solve
        fd = torch.tensor(f, device="cuda")
        for prec in ("f64", "f32_refine"):
            ud = torch.zeros_like(fd)
            # alternating tweed / wireframe (Sec. 3): fast on every grid here
            res = g.solve(ud, fd, smoother="alt_tw", nu1=1, nu2=1, precision=prec, tol=1e-8, max_cycles=60,
                          max_outer=30)
            calls += 1
            assert res.status == mg.OK, (nx, ny, kind, prec, res.status, res.cycles, res.rel_res)
    # 3D tweed and wireframe solves
    z = I.wall_coords(16, I.c_for_ratio(16, 20.0))
    zc = I.coords(16, "centre", ratio=5.0)
    f3 = rng.standard_normal((17, 17, 17))
    for coords, sm in ((z, "tweed"), (zc, "wireframe")):
        g3 = mg.Grid(coords, coords, coords)
        u3 = torch.zeros(f3.shape, dtype=torch.float64, device="cuda")
        res = g3.solve(u3, torch.tensor(f3, device="cuda"), smoother=sm, nu1=2, nu2=2, tol=1e-10)
        calls += 1
        assert res.status == mg.OK, (sm, res.status, res.cycles, res.rel_res)
    # the 3D tiled tweed path on a 64^3 level, both colours, FP64 and FP32
    x3 = I.wall_coords(64, I.c_for_ratio(64, 50.0))
    g3, P3 = mg.Grid(x3, x3, x3), oracle.Problem3(x3, x3, x3)
    g3.set_line_path(0, "tweed", "f64", "tiled")
    u0, f0 = rng.standard_normal(P3.shape()), rng.standard_normal(P3.shape())
    for colour in (0, 1):
        ref = P3.colour_pass(u0.copy(), f0, colour)
        for dt, tol in (("f64", 1e-10), ("f32", 2e-3)):
            tdt = torch.float64 if dt == "f64" else torch.float32
            ud = torch.tensor(u0, dtype=tdt, device="cuda")
            g3.colour_pass(ud, torch.tensor(f0, dtype=tdt, device="cuda"), "tweed", colour)
            calls += 1
            got = ud.double().cpu().numpy()
            assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max()), ("3d tiled", colour, dt)
    # a batch of two problems
    xs = [I.wall_coords(64, 2.0), I.wall_coords(128, 3.0)]
    bg = [mg.Grid(x, x) for x in xs]
    fs = [torch.tensor(rng.standard_normal((len(x), len(x))), device="cuda") for x in xs]
    us = [torch.zeros_like(fb) for fb in fs]
    out = mg.Batch(bg).solve(us, fs, smoother="tweed", nu1=1, nu2=1, tol=1e-10, precision="f32_refine")
    calls += 1
    assert all(r.status == mg.OK for r in out), [(r.status, r.cycles) for r in out]
    torch.cuda.synchronize()
    w = lib.mg_check_word()
    assert w == CHECKED, hex(w)
    print(f"checked ok {calls}")


if __name__ == "__main__":
    main()
