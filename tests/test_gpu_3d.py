"""3D grids (Sec. 7) through the C ABI against the 3D oracle: tweed and
wireframe colour passes on every smoothed level (FP64 to 1e-10, FP32 to the
FP32 smoothing tolerance), the tiled tweed path of the large levels, the 7-point defect, full-weighting restriction,
trilinear prolongation and coarsest solve, the FP64 solve history per cycle
(1e-12 on the relative residual, 1 % on the convergence factor) and FP32
cycles with FP64 refinement to 1e-10."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GRIDS3 = [  # (nx, ny, nz, kind, ratio)
    (8, 8, 8, "wall", 20.0),
    (16, 12, 10, "wall", 50.0),
    (32, 32, 32, "wall", 200.0),
    (24, 16, 32, "centre", 5.0),
]


def coords3(nx, ny, nz, kind, ratio):
    return tuple(I.coords(n, kind, ratio=ratio) for n in (nx, ny, nz))


def pair(mg, oracle_mod, grid):
    xyz = coords3(*grid)
    return mg.Grid(*xyz), oracle_mod.Problem3(*xyz)


def cuda(a, dtype="f64"):
    import torch
    return torch.tensor(a, dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("smoother", ["tweed", "wireframe"])
@pytest.mark.parametrize("grid", GRIDS3, ids=lambda t: f"{t[0]}x{t[1]}x{t[2]}-{t[3]}")
def test_colour_pass_3d(mg, oracle_mod, grid, smoother):
    g, P = pair(mg, oracle_mod, grid)
    assert g.nlev == P.nlev
    rng = np.random.default_rng(11)
    for lev in range(g.nlev - 1):
        assert g.shape(lev) == P.shape(lev)
        u0, f = rng.standard_normal(P.shape(lev)), rng.standard_normal(P.shape(lev))
        for colour in (0, 1):
            ref = P.colour_pass(u0.copy(), f, colour, lev, smoother=smoother)
            ud = cuda(u0)
            g.colour_pass(ud, cuda(f), smoother, colour, level=lev)
            assert rel_err(host(ud), ref) <= 1e-10, (lev, colour, rel_err(host(ud), ref))
        # FP32: one relaxation on FP32-rounded data
        u32 = u0.astype(np.float32).astype(np.float64)
        f32 = f.astype(np.float32).astype(np.float64)
        ref = P.smooth(u32.copy(), f32, lev, smoother=smoother)
        ud = cuda(u32, "f32")
        g.smooth(ud, cuda(f32, "f32"), smoother, 1, level=lev)
        assert rel_err(host(ud), ref) <= 2e-4, (lev, rel_err(host(ud), ref))


TILED3 = [(64, 64, 64, "wall", 200.0), (64, 96, 128, "centre", 10.0), (128, 64, 96, "wall", 50.0)]


@pytest.mark.parametrize("grid", TILED3, ids=lambda t: f"{t[0]}x{t[1]}x{t[2]}-{t[3]}")
def test_tiled_tweed_pass_3d(mg, oracle_mod, grid):
    """The 3D tiled tweed path (32 chunks of parallel legs per warp, one per
    lane) on every level whose sides are all at least 64 intervals, selected
    with mg_set_line_path (the built-in rule takes it from 256 intervals on):
    each colour pass against the oracle (FP64 to 1e-10; FP32 on FP32-rounded
    data to 2e-4), and against the same pass on the warp path (FP64, 1e-10)."""
    g, P = pair(mg, oracle_mod, grid)
    rng = np.random.default_rng(15)
    tiled = [lev for lev in range(g.nlev - 1) if min(P.dims(lev)) >= 64]
    assert tiled
    for lev in tiled:
        assert g.line_path(lev, "tweed", "f64")[0] == "warp"
        g.set_line_path(lev, "tweed", "f64", "tiled")
        assert g.line_path(lev, "tweed", "f64")[0] == "tiled"
        u0, f = rng.standard_normal(P.shape(lev)), rng.standard_normal(P.shape(lev))
        u32 = u0.astype(np.float32).astype(np.float64)
        f32 = f.astype(np.float32).astype(np.float64)
        for colour in (0, 1):
            ref = P.colour_pass(u0.copy(), f, colour, lev)
            ud = cuda(u0)
            g.colour_pass(ud, cuda(f), "tweed", colour, level=lev)
            got = host(ud)
            assert rel_err(got, ref) <= 1e-10, (lev, colour, rel_err(got, ref))
            g.set_line_path(lev, "tweed", "f64", "warp")
            uw = cuda(u0)
            g.colour_pass(uw, cuda(f), "tweed", colour, level=lev)
            g.set_line_path(lev, "tweed", "f64", "tiled")
            assert rel_err(host(uw), got) <= 1e-10
            ref32 = P.colour_pass(u32.copy(), f32, colour, lev)
            u3 = cuda(u32, "f32")
            g.colour_pass(u3, cuda(f32, "f32"), "tweed", colour, level=lev)
            assert rel_err(host(u3), ref32) <= 2e-4, (lev, colour, rel_err(host(u3), ref32))


def test_tiled_path_requests_3d(mg):
    """mg_set_line_path on 3D grids: the tiled path exists for tweed on levels
    whose sides are all at least 64 intervals; wireframe has the warp path
    alone; the coarsest level has no passes."""
    g = mg.Grid(*coords3(64, 64, 64, "wall", 20.0))
    g.set_line_path(0, "tweed", "f32", "tiled")
    assert g.line_path(0, "tweed", "f32")[0] == "tiled"
    with pytest.raises(mg.MGError) as e:
        g.set_line_path(1, "tweed", "f32", "tiled")  # 32^3
    assert e.value.status == mg.ERR_UNSUPPORTED
    with pytest.raises(mg.MGError) as e:
        g.set_line_path(0, "wireframe", "f32", "tiled")
    assert e.value.status == mg.ERR_UNSUPPORTED
    with pytest.raises(mg.MGError) as e:
        g.set_line_path(g.nlev - 1, "tweed", "f32", "warp")
    assert e.value.status == mg.ERR_INVALID_ARG
    assert g.line_path(1, "tweed", "f32")[0] == "warp"


@pytest.mark.parametrize("grid", GRIDS3[1:], ids=lambda t: f"{t[0]}x{t[1]}x{t[2]}-{t[3]}")
def test_transfers_and_coarse_3d(mg, oracle_mod, grid):
    import torch
    g, P = pair(mg, oracle_mod, grid)
    rng = np.random.default_rng(12)
    for lev in range(g.nlev - 1):
        u, f = rng.standard_normal(P.shape(lev)), rng.standard_normal(P.shape(lev))
        d_ref = P.residual(u, f, lev)
        d = torch.empty_like(cuda(u))
        g.residual(cuda(u), cuda(f), d, level=lev)
        assert rel_err(host(d), d_ref) <= 1e-12
        fc = torch.zeros(P.shape(lev + 1), dtype=torch.float64, device="cuda")
        uc = torch.ones_like(fc)
        g.residual_restrict(cuda(u), cuda(f), fc, uc, level=lev)
        fc_ref = P.restrict(d_ref, lev)
        inner = (slice(1, -1),) * 3
        assert rel_err(host(fc)[inner], fc_ref[inner]) <= 1e-12
        assert (host(uc)[inner] == 0).all()
        ucr = rng.standard_normal(P.shape(lev + 1))
        ucr[0, :, :] = ucr[-1, :, :] = 0; ucr[:, 0, :] = ucr[:, -1, :] = 0; ucr[:, :, 0] = ucr[:, :, -1] = 0
        ud = cuda(u)
        g.prolong_add(cuda(ucr), ud, level=lev)
        assert rel_err(host(ud), P.prolong_add(ucr, u.copy(), lev)) <= 1e-13
    lc = g.nlev - 1
    u, f = rng.standard_normal(P.shape(lc)), rng.standard_normal(P.shape(lc))
    ref = P.direct_solve(u.copy(), f, lc)
    ud = cuda(u)
    g.coarse_solve(ud, cuda(f))
    assert rel_err(host(ud), ref) <= 1e-10


@pytest.mark.parametrize("grid,smoother", [((32, 32, 32, "wall", 200.0), "tweed"), ((16, 12, 10, "wall", 50.0), "tweed"),
                                           ((64, 64, 64, "wall", 200.0), "tweed"),
                                           ((32, 32, 32, "centre", 10.0), "wireframe"),
                                           ((24, 16, 32, "centre", 5.0), "wireframe"),
                                           ((32, 32, 32, "wall", 50.0), "alt_tw")],
                         ids=lambda t: f"{t[0]}x{t[1]}x{t[2]}-{t[3]}" if isinstance(t, tuple) else t)
def test_solve_history_3d(mg, oracle_mod, grid, smoother):
    """FP64 V(2,2) cycles: the relative residual after every cycle within
    1e-12 of the oracle's and the convergence factor within 1 %."""
    g, P = pair(mg, oracle_mod, grid)
    if min(grid[:3]) >= 64 and smoother == "tweed":
        g.set_line_path(0, "tweed", "f64", "tiled")  # the 3D tiled path inside the cycles
    rng = np.random.default_rng(13)
    f = rng.standard_normal(P.shape())
    bnd = rng.standard_normal(P.shape())
    bnd[1:-1, 1:-1, 1:-1] = 0.0
    u_ref = bnd.copy()
    hist_ref = P.solve(u_ref, f, nu1=2, nu2=2, tol=1e-10, max_cycles=60, smoother=smoother)
    ud = cuda(bnd)
    res = g.solve(ud, cuda(f), smoother=smoother, nu1=2, nu2=2, tol=1e-10, max_cycles=60, precision="f64")
    assert res.status == mg.OK
    assert res.cycles == len(hist_ref) - 1
    assert np.abs(np.asarray(res.history) - hist_ref).max() <= 1e-12
    k = len(hist_ref) - 1
    fac_ref = (hist_ref[-1] / hist_ref[0]) ** (1.0 / k)
    assert abs(res.conv_factor - fac_ref) <= 0.01 * fac_ref
    assert rel_err(host(ud), u_ref) <= 1e-8


@pytest.mark.parametrize("smoother,kind,ratio,path", [("tweed", "wall", 200.0, "warp"), ("tweed", "wall", 200.0, "tiled"),
                                                      ("wireframe", "centre", 10.0, "warp")])
def test_f32_refine_3d(mg, oracle_mod, smoother, kind, ratio, path):
    g, P = pair(mg, oracle_mod, (64, 64, 64, kind, ratio))
    if path == "tiled":
        g.set_line_path(0, "tweed", "f32", "tiled")
    f = np.random.default_rng(14).standard_normal(P.shape())
    ud = cuda(np.zeros(P.shape()))
    res = g.solve(ud, cuda(f), smoother=smoother, nu1=2, nu2=2, tol=1e-10, precision="f32_refine", max_outer=40,
                  max_cycles=400)
    assert res.status == mg.OK and res.rel_res <= 1e-10
    d = P.residual(host(ud), f)
    assert np.linalg.norm(d[1:-1, 1:-1, 1:-1]) / np.linalg.norm(f[1:-1, 1:-1, 1:-1]) <= 1.5e-10


def test_3d_unsupported_requests(mg):
    import torch
    xyz = coords3(8, 8, 8, "wall", 10.0)
    g = mg.Grid(*xyz)
    assert g.dim == 3 and mg.load().mg_grid_dim(g.h) == 3
    u = torch.zeros(g.shape(), dtype=torch.float64, device="cuda")
    for sm in ("zebra_x", "checkerboard"):
        with pytest.raises(mg.MGError) as e:
            g.colour_pass(u, u, sm, 0)
        assert e.value.status == mg.ERR_UNSUPPORTED
    for sm in ("zebra_y", "alt_zebra"):
        with pytest.raises(mg.MGError) as e:
            g.solve(u, u.clone() + 1, smoother=sm)
        assert e.value.status == mg.ERR_UNSUPPORTED
    with pytest.raises(mg.MGError) as e:
        mg.Batch([g])
    assert e.value.status == mg.ERR_UNSUPPORTED


@pytest.mark.parametrize("dims", [(16, 16, 16), (24, 16, 32), (64, 48, 32)])
def test_wireframe_skeleton_and_rings_3d(mg, oracle_mod, dims):
    """A red then a black wireframe pass on the finest level of grids with
    many cuboid skeletons and rings of every size: FP64 against the oracle."""
    g, P = pair(mg, oracle_mod, (*dims, "centre", 20.0))
    rng = np.random.default_rng(15)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())
    ref = u0.copy()
    ud = cuda(u0)
    for colour in (0, 1):
        ref = P.colour_pass(ref, f, colour, smoother="wireframe")
        g.colour_pass(ud, cuda(f), "wireframe", colour)
    assert rel_err(host(ud), ref) <= 1e-10
