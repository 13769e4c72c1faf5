"""Every line-solve path (warp sequences of each shape, cluster, tiled, CTA)
against the oracle on every level where the blocks fit it, and the autotuner
that picks among them (mg_set_line_path / mg_get_line_path / mg_autotune).

The paths differ only in how a colour pass is spread over the GPU; each must
give the exact block solves of Sec. 3, so the FP64 tolerance is the one of the
plain colour-pass parity tests (1e-10 relative to max |u|)."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WARP_KS = [1, 2, 4, 8, 16]


def coords(n, kind, c):
    return {"wall": lambda n: I.wall_coords(n, c), "centre": lambda n: I.centre_coords(n, c)}[kind](n)


def cuda(a, dtype):
    import torch
    return torch.tensor(a, dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def pass_cases(g, level, smoother, dtype, mg):
    """(label, path, k) for every path that level takes, one per distinct shape."""
    out, seen = [], set()
    for path, ks in (("warp", WARP_KS), ("cluster", [0]), ("tiled", [0]), ("cta", [0])):
        for k in ks:
            try:
                g.set_line_path(level, smoother, dtype, path, k)
            except mg.MGError as e:
                assert e.status == mg.ERR_UNSUPPORTED
                continue
            shape = g.line_path(level, smoother, dtype)
            assert shape[0] == path
            if shape in seen:
                continue
            seen.add(shape)
            out.append((f"{path}{shape[1:] if path == 'warp' else ''}", path, k))
    g.set_line_path(level, smoother, dtype, "auto")
    return out


@pytest.mark.parametrize("grid,smoother", [
    ((64, 64, "wall", 3.0), "tweed"),
    ((96, 136, "centre", 2.0), "wireframe"),
    ((272, 512, "centre", 1.2), "tweed"),     # T-blocks and lines
    ((200, 72, "wall", 2.5), "zebra_x"),
    ((1024, 1024, "wall", 3.0), "tweed"),     # centre cross of 2045 nodes; tiled path at level 0
    ((1024, 1024, "wall", 3.0), "zebra_y"),
], ids=lambda v: f"{v[0]}x{v[1]}-{v[2]}" if isinstance(v, tuple) else v)
def test_every_path_matches_oracle_f64(mg, oracle_mod, grid, smoother):
    nx, ny, kind, c = grid
    x, y = coords(nx, kind, c), coords(ny, kind, c)
    g, P = mg.Grid(x, y), oracle_mod.Problem(x, y)
    rng = np.random.default_rng(7)
    tested = 0
    for level in range(g.nlev - 1):
        u0 = rng.standard_normal(P.shape(level))
        f = rng.standard_normal(P.shape(level))
        refs = [P.colour_pass(u0.copy(), f, smoother, colour, level) for colour in (0, 1)]
        for label, path, k in pass_cases(g, level, smoother, "f64", mg):
            g.set_line_path(level, smoother, "f64", path, k)
            for colour in (0, 1):
                ud = cuda(u0, "f64")
                g.colour_pass(ud, cuda(f, "f64"), smoother, colour, level=level)
                err = rel_err(host(ud), refs[colour])
                assert err <= 1e-10, (level, label, colour, err)
            tested += 1
        g.set_line_path(level, smoother, "f64", "auto")
    assert tested >= 2 * (g.nlev - 1)


def test_f32_warp_shapes(mg, oracle_mod):
    """FP32 passes of every warp shape of a 1025^2 level match the FP64 oracle
    on FP32-rounded data to the FP32 tolerance of the smoothing tests."""
    x = coords(1024, "wall", 3.0)
    g, P = mg.Grid(x, x), oracle_mod.Problem(x, x)
    rng = np.random.default_rng(8)
    u0 = rng.standard_normal(P.shape(0)).astype(np.float32).astype(np.float64)
    f = rng.standard_normal(P.shape(0)).astype(np.float32).astype(np.float64)
    refs = [P.colour_pass(u0.copy(), f, "tweed", colour, 0) for colour in (0, 1)]
    cases = pass_cases(g, 0, "tweed", "f32", mg)
    assert {c[1] for c in cases} == {"warp", "cluster", "tiled", "cta"}
    for label, path, k in cases:
        g.set_line_path(0, "tweed", "f32", path, k)
        for colour in (0, 1):
            ud = cuda(u0, "f32")
            g.colour_pass(ud, cuda(f, "f32"), "tweed", colour, level=0)
            assert rel_err(host(ud), refs[colour]) <= 2e-4, (label, colour)


@pytest.mark.parametrize("grid,smoother", [
    ((1024, 1024, "wall", 3.0), "tweed"),     # L-blocks over up to 4 CTAs, the centre cross compact
    ((1024, 1024, "wall", 3.0), "zebra_x"),   # lines of 32 chunks over 2 CTAs
    ((1024, 1024, "wall", 3.0), "zebra_y"),
    ((2048, 1024, "wall", 2.0), "tweed"),     # T-blocks (compact) and wall-to-wall lines
    ((1088, 1600, "centre", 1.5), "tweed"),   # ragged chunks and tiles, T-blocks
], ids=lambda v: f"{v[0]}x{v[1]}-{v[2]}" if isinstance(v, tuple) else v)
def test_cluster_pass_f32(mg, oracle_mod, grid, smoother):
    """The cluster path's FP32 colour passes against the FP64 oracle on
    FP32-rounded data (the FP32 smoothing tolerance), and against the FP32
    tiled path, which solves the same blocks in another grouping; the
    other colour and the boundary stay untouched bit for bit."""
    nx, ny, kind, c = grid
    x, y = coords(nx, kind, c), coords(ny, kind, c)
    g, P = mg.Grid(x, y), oracle_mod.Problem(x, y)
    rng = np.random.default_rng(9)
    u0 = rng.standard_normal(P.shape(0)).astype(np.float32).astype(np.float64)
    f = rng.standard_normal(P.shape(0)).astype(np.float32).astype(np.float64)
    for colour in (0, 1):
        ref = P.colour_pass(u0.copy(), f, smoother, colour, 0)
        got = {}
        for path in ("cluster", "tiled"):
            g.set_line_path(0, smoother, "f32", path)
            assert g.line_path(0, smoother, "f32")[0] == path
            ud = cuda(u0, "f32")
            g.colour_pass(ud, cuda(f, "f32"), smoother, colour, level=0)
            got[path] = host(ud)
        g.set_line_path(0, smoother, "f32", "auto")
        same = ref == u0
        assert np.array_equal(got["cluster"][same], u0[same])
        assert rel_err(got["cluster"], ref) <= 2e-4, (colour, rel_err(got["cluster"], ref))
        assert rel_err(got["cluster"], got["tiled"]) <= 2e-4


def test_default_paths_and_unsupported(mg):
    x = coords(1024, "wall", 3.0)
    g = mg.Grid(x, x)
    # built-in rule, reported for colour 0 (odd levels k of max(d_x, d_y)):
    # its largest blocks, the L-blocks of k = 511 with 1021 nodes, fit 8
    # warps of the preferred 4 nodes per thread
    assert g.line_path(0, "tweed", "f32") == ("warp", 4, 8)
    assert g.line_path(0, "tweed", "f64") == ("warp", 4, 8)
    # wireframe rings of 4085 nodes: FP64 warp sequences hold at most 2048
    with pytest.raises(mg.MGError) as e:
        g.set_line_path(0, "wireframe", "f64", "warp")
    assert e.value.status == mg.ERR_UNSUPPORTED
    assert g.line_path(0, "wireframe", "f64")[0] == "cta"
    # no tiled lists below 1024 intervals, nor for wireframe; no cluster
    # path there either, nor in FP64
    small = mg.Grid(coords(64, "wall", 3.0), coords(64, "wall", 3.0))
    for grid, lev, sm, dt, path in ((small, 0, "tweed", "f32", "tiled"), (g, 0, "wireframe", "f32", "tiled"),
                                    (small, 0, "tweed", "f32", "cluster"), (g, 0, "wireframe", "f32", "cluster"),
                                    (g, 0, "tweed", "f64", "cluster")):
        with pytest.raises(mg.MGError) as e:
            grid.set_line_path(lev, sm, dt, path)
        assert e.value.status == mg.ERR_UNSUPPORTED
    with pytest.raises(mg.MGError) as e:
        g.set_line_path(0, "tweed", "f32", "warp", 3)
    assert e.value.status == mg.ERR_INVALID_ARG


def test_autotune_then_solve(mg, oracle_mod):
    """The tuned grid still solves to tolerance, a second grid of the same
    size takes the remembered choices without timing, and the paths chosen
    are ones the level supports."""
    import torch
    n = 256
    x = coords(n, "wall", 3.0)
    g = mg.Grid(x, x)
    times = g.autotune("tweed", "f32", reps=6)
    assert len(times) == g.nlev and times[-1] == 0.0
    assert all(t > 0.0 for t in times[:-1])
    chosen = [g.line_path(level, "tweed", "f32") for level in range(g.nlev - 1)]
    g2 = mg.Grid(x, x)
    times2 = g2.autotune("tweed", "f32", reps=0)
    assert times2 == times
    assert [g2.line_path(level, "tweed", "f32") for level in range(g2.nlev - 1)] == chosen
    f = torch.tensor(I.rhs_gaussian(n + 1, n + 1, 3), device="cuda")
    u = torch.zeros_like(f)
    p = mg.default_params(smoother="tweed", nu1=1, nu2=1, precision="f32_refine", tol=1e-10, max_outer=30)
    res = g.solve(u, f, p)
    assert res.status == mg.OK and res.rel_res <= 1e-10
    P = oracle_mod.Problem(x, x)
    d, fh = P.residual(host(u), host(f)), host(f)
    assert np.linalg.norm(d[1:-1, 1:-1]) / np.linalg.norm(fh[1:-1, 1:-1]) <= 1.5e-10
