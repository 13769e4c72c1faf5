"""GPU parity: every kernel of the CUDA path, called through the C ABI, against
the CPU oracle on the same seeded inputs.

Tolerances:
  FP64, single kernels: |gpu - oracle| <= 1e-10 * max|oracle| -- both sides solve
      the same blocks exactly with different elimination orders; the blocks of
      these test grids have condition numbers below ~1e4, so rounding
      differences stay near 1e-12.
  FP64 cycles: per-cycle relative residual within 1e-12 absolute (the solver
      contract), measured convergence factor within 1 %.
  FP32 kernels: |gpu - oracle| <= 2e-4 * max|oracle| (FP32 rounding of the
      coefficients and of the elimination, amplified by block condition
      numbers up to ~1e3 on the FP32 test grids).
"""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GRIDS = [
    # (nx, ny, kind, c)  -- several chunks per run, ragged tails, rectangles,
    # the minimal grids
    (2, 2, "uniform", 0.0),
    (4, 2, "uniform", 0.0),
    (2, 6, "uniform", 0.0),
    (8, 8, "wall", 1.5),
    (16, 10, "centre", 1.5),
    (12, 30, "wall", 2.0),
    (64, 64, "wall", 3.0),
    (96, 136, "centre", 2.0),
    (200, 72, "wall", 2.5),
    (256, 256, "wall", 3.043),
    (320, 256, "wall", 2.0),      # T-blocks and lines
    (272, 512, "centre", 1.2),    # rows longer than columns
    (1024, 1024, "wall", 3.0),    # tiled line path (both sides >= 1024): L-blocks, centre cross
    (1152, 1024, "centre", 1.2),  # tiled: T-blocks, straight lines, ragged last tiles
]
BASE_SMOOTHERS = ["checkerboard", "zebra_x", "zebra_y", "tweed", "wireframe"]


def coords(n, kind, c):
    return {"uniform": I.uniform_coords, "wall": lambda n: I.wall_coords(n, c),
            "centre": lambda n: I.centre_coords(n, c)}[kind](n)


def setup_pair(mg, oracle_mod, nx, ny, kind, c):
    x, y = coords(nx, kind, c), coords(ny, kind, c)
    return mg.Grid(x, y), oracle_mod.Problem(x, y)


def cuda(a, dtype="f64"):
    import torch
    return torch.tensor(a, dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_exports(mg):
    lib = mg.load()
    for name in mg.EXPORTS:
        assert hasattr(lib, name)


def test_levels_match_oracle(mg, oracle_mod):
    for nx, ny, kind, c in GRIDS:
        g, P = setup_pair(mg, oracle_mod, nx, ny, kind, c)
        assert g.nlev == P.nlev
        for l in range(g.nlev):
            assert g.shape(l) == P.shape(l)


@pytest.mark.parametrize("grid", GRIDS, ids=lambda t: f"{t[0]}x{t[1]}-{t[2]}")
@pytest.mark.parametrize("smoother", BASE_SMOOTHERS)
def test_colour_pass_f64(mg, oracle_mod, grid, smoother):
    g, P = setup_pair(mg, oracle_mod, *grid)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal(P.shape())          # boundary values included
    f = rng.standard_normal(P.shape())
    for colour in (0, 1):
        ref = P.colour_pass(u0.copy(), f, smoother, colour)
        ud = cuda(u0)
        g.colour_pass(ud, cuda(f), smoother, colour)
        got = host(ud)
        assert np.array_equal(got[0, :], u0[0, :]) and np.array_equal(got[:, -1], u0[:, -1])
        assert rel_err(got, ref) <= 1e-10, (grid, smoother, colour, rel_err(got, ref))


@pytest.mark.parametrize("grid", GRIDS[3:], ids=lambda t: f"{t[0]}x{t[1]}-{t[2]}")
@pytest.mark.parametrize("smoother", BASE_SMOOTHERS + ["alt_zebra", "alt_tw"])
def test_smooth_f32(mg, oracle_mod, grid, smoother):
    g, P = setup_pair(mg, oracle_mod, *grid)
    rng = np.random.default_rng(2)
    u0 = rng.standard_normal(P.shape()).astype(np.float32).astype(np.float64)
    f = rng.standard_normal(P.shape()).astype(np.float32).astype(np.float64)
    ref = P.smooth(u0.copy(), f, smoother, 1)
    ud = cuda(u0, "f32")
    g.smooth(ud, cuda(f, "f32"), smoother, 1)
    assert rel_err(host(ud), ref) <= 2e-4, rel_err(host(ud), ref)


@pytest.mark.parametrize("smoother", ["zebra_x", "zebra_y", "tweed", "alt_zebra"])
def test_smooth_f32_long_lines(mg, oracle_mod, smoother):
    """4096 x 1024 intervals, level 0 on the tiled path: the zebra-x lines have 4095
    nodes, 128 chunks, more than the 64 a leg may have for the FP32 couple
    with setup-time pivots, so that list keeps the plain couple; the zebra-y
    lines (32 chunks) and the tweed blocks (L-blocks, T-blocks, straight
    lines) take the pivots from setup.  Each against the oracle as
    test_smooth_f32."""
    g, P = setup_pair(mg, oracle_mod, 4096, 1024, "wall", 2.0)
    for sm in (("zebra_x", "zebra_y") if smoother == "alt_zebra" else (smoother,)):
        g.set_line_path(0, sm, "f32", "tiled")
        assert g.line_path(0, sm, "f32")[0] == "tiled"
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(P.shape()).astype(np.float32).astype(np.float64)
    f = rng.standard_normal(P.shape()).astype(np.float32).astype(np.float64)
    ref = P.smooth(u0.copy(), f, smoother, 1)
    ud = cuda(u0, "f32")
    g.smooth(ud, cuda(f, "f32"), smoother, 1)
    assert rel_err(host(ud), ref) <= 2e-4, rel_err(host(ud), ref)


@pytest.mark.parametrize("grid", GRIDS[3:], ids=lambda t: f"{t[0]}x{t[1]}-{t[2]}")
@pytest.mark.parametrize("restriction", [0, 1])
def test_residual_restrict_prolong(mg, oracle_mod, grid, restriction):
    g, P = setup_pair(mg, oracle_mod, *grid)
    if P.nlev < 2:
        pytest.skip("single level")
    rng = np.random.default_rng(3)
    u = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    d_ref = P.residual(u, f)
    fc_ref = P.restrict(d_ref, restriction)
    ud, fd = cuda(u), cuda(f)
    dd = cuda(np.full(P.shape(), np.nan))
    g.residual(ud, fd, dd)
    assert rel_err(host(dd), d_ref) <= 1e-12
    fc = cuda(np.full(P.shape(1), 7.0))
    uc = cuda(np.full(P.shape(1), 9.0))
    uc_b = host(uc)
    g.residual_restrict(ud, fd, fc, uc, restriction=restriction)
    got = host(fc)
    assert rel_err(got[1:-1, 1:-1], fc_ref[1:-1, 1:-1]) <= 1e-12
    ucg = host(uc)
    assert np.all(ucg[1:-1, 1:-1] == 0.0) and np.array_equal(ucg[0, :], uc_b[0, :])
    v = I.random_field(*P.shape(1), seed=5)
    ref = P.prolong_add(v, u.copy())
    g.prolong_add(cuda(v), ud)
    assert rel_err(host(ud), ref) <= 1e-14


@pytest.mark.parametrize("grid", GRIDS, ids=lambda t: f"{t[0]}x{t[1]}-{t[2]}")
def test_coarse_solve(mg, oracle_mod, grid):
    g, P = setup_pair(mg, oracle_mod, *grid)
    lev = P.nlev - 1
    rng = np.random.default_rng(4)
    u = rng.standard_normal(P.shape(lev))
    f = rng.standard_normal(P.shape(lev))
    ref = P.direct_solve(u, f, lev)
    ud = cuda(u)
    g.coarse_solve(ud, cuda(f))
    assert rel_err(host(ud), ref) <= 1e-11


@pytest.mark.parametrize("grid", GRIDS[3:], ids=lambda t: f"{t[0]}x{t[1]}-{t[2]}")
@pytest.mark.parametrize("smoother,nu,cycle,restriction",
                         [("tweed", (2, 2), "V", 1), ("wireframe", (1, 1), "V", 1), ("checkerboard", (1, 2), "W", 0),
                          ("alt_zebra", (1, 1), "V", 1), ("alt_tw", (2, 1), "W", 1)])
def test_cycle_f64(mg, oracle_mod, grid, smoother, nu, cycle, restriction):
    g, P = setup_pair(mg, oracle_mod, *grid)
    rng = np.random.default_rng(6)
    u0 = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    ref = P.cycle(u0.copy(), f, smoother, nu[0], nu[1], 1 if cycle == "V" else 2, restriction)
    ud = cuda(u0)
    g.vcycle(ud, cuda(f), smoother=smoother, nu1=nu[0], nu2=nu[1], cycle=cycle, restriction=restriction)
    assert rel_err(host(ud), ref) <= 1e-10


def config1():
    """65^2 nodes, wall clustering with spacing ratio 100, manufactured
    solution plus 1e-3 uniform noise (seed 0), V(2,2) tweed, full weighting."""
    n = 64
    x = I.wall_coords(n, I.c_for_ratio(n, 100.0))
    _, f = I.manufactured(x, x, noise=1e-3, seed=0)
    return x, f


def test_config1_solve_history_f64(mg, oracle_mod):
    x, f = config1()
    P = oracle_mod.Problem(x, x)
    u_ref, hist_ref, _ = P.solve(np.zeros_like(f), f, "tweed", 2, 2, tol=1e-10)
    g = mg.Grid(x, x)
    ud = cuda(np.zeros_like(f))
    res = g.solve(ud, cuda(f), smoother="tweed", nu1=2, nu2=2, tol=1e-10)
    assert res.status == mg.OK
    assert len(res.history) == len(hist_ref)
    assert np.abs(res.history - hist_ref).max() <= 1e-12
    k = len(hist_ref) - 1
    fac_ref = (hist_ref[-1] / hist_ref[0]) ** (1 / k)
    assert res.conv_factor == pytest.approx(fac_ref, rel=0.01)
    assert rel_err(host(ud), u_ref) <= 1e-10


@pytest.mark.parametrize("smoother,kind,c", [("tweed", "wall", 3.0), ("wireframe", "centre", 1.5),
                                             ("alt_zebra", "wall", 3.0), ("checkerboard", "uniform", 0.0)])
def test_solve_history_other_smoothers(mg, oracle_mod, smoother, kind, c):
    x = coords(128, kind, c)
    f = I.rhs_gaussian(129, 129, seed=1)
    P = oracle_mod.Problem(x, x)
    _, hist_ref, _ = P.solve(np.zeros_like(f), f, smoother, 1, 1, tol=1e-10, max_cycles=40)
    g = mg.Grid(x, x)
    res = g.solve(cuda(np.zeros_like(f)), cuda(f), smoother=smoother, nu1=1, nu2=1, tol=1e-10, max_cycles=40)
    assert len(res.history) == len(hist_ref)
    assert np.abs(res.history - hist_ref).max() <= 1e-12


def test_f32_refine_reaches_tolerance(mg, oracle_mod):
    x, f = config1()
    P = oracle_mod.Problem(x, x)
    u_ref, _, _ = P.solve(np.zeros_like(f), f, "tweed", 2, 2, tol=1e-12)
    g = mg.Grid(x, x)
    ud = cuda(np.zeros_like(f))
    res = g.solve(ud, cuda(f), smoother="tweed", nu1=2, nu2=2, tol=1e-10, precision="f32_refine")
    assert res.status == mg.OK and res.rel_res <= 1e-10
    assert res.outer_iters <= 4
    # both solutions satisfy the same tolerance; their distance is bounded by it
    assert rel_err(host(ud), u_ref) <= 1e-8


def test_boundary_data_respected(mg, oracle_mod):
    """Non-zero Dirichlet data: the solve equals the dense-LU solution."""
    x = I.wall_coords(8, 1.5)
    y = I.wall_coords(6, 1.5)
    P = oracle_mod.Problem(x, y)
    rng = np.random.default_rng(9)
    gdat = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    ref = P.direct_solve(gdat, f)
    g = mg.Grid(x, y)
    for prec in ("f64", "f32_refine"):
        ud = cuda(gdat)
        res = g.solve(ud, cuda(f), precision=prec, tol=1e-12, smoother="tweed")
        assert res.status == mg.OK
        assert rel_err(host(ud), ref) <= 1e-10


def test_adjoint_identity(mg, oracle_mod):
    """<L v, lambda> = <v, rhs> for zero-boundary v when L^T lambda = rhs (L
    applied by the oracle; independent of the scaling used inside)."""
    x = I.wall_coords(64, 2.5)
    y = I.centre_coords(32, 1.2)
    P = oracle_mod.Problem(x, y)
    rhs = I.random_field(*P.shape(), seed=12)
    g = mg.Grid(x, y)
    lam = cuda(np.zeros(P.shape()))
    res = g.solve_adjoint(lam, cuda(rhs), tol=1e-12, smoother="tweed")
    assert res.status == mg.OK
    lam_h = host(lam)
    for s in range(3):
        v = I.random_field(*P.shape(), seed=20 + s)
        lhs = np.sum(P.apply(v) * lam_h)
        rhs_ = np.sum(v * rhs)
        assert lhs == pytest.approx(rhs_, rel=1e-8)


def test_errors_are_status_codes(mg):
    import ctypes
    lib = mg.load()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 2)(1, 8)
    x = np.linspace(0, 1, 2)
    y = np.linspace(0, 1, 9)
    co = (ctypes.c_void_p * 2)(x.ctypes.data, y.ctypes.data)
    assert lib.mg_setup_grid(ctypes.byref(h), 2, n, co, 3, None) == mg.ERR_SIZE
    n = (ctypes.c_int64 * 2)(8, 8)
    xb = np.linspace(0, 1, 9)
    xb[4] = xb[3]
    co = (ctypes.c_void_p * 2)(xb.ctypes.data, xb.ctypes.data)
    assert lib.mg_setup_grid(ctypes.byref(h), 2, n, co, 3, None) == mg.ERR_SIZE
    n3 = (ctypes.c_int64 * 3)(8, 8, 8)
    co3 = (ctypes.c_void_p * 3)(xb.ctypes.data, xb.ctypes.data, xb.ctypes.data)
    assert lib.mg_setup_grid(ctypes.byref(h), 3, n3, co3, 3, None) == mg.ERR_SIZE
    assert lib.mg_setup_grid(ctypes.byref(h), 4, n3, co3, 3, None) == mg.ERR_INVALID_ARG
    g = mg.Grid(np.linspace(0, 1, 9), np.linspace(0, 1, 9))
    assert lib.mg_smooth(g.h, 5, 4, None, None, 1, 0, None) == mg.ERR_INVALID_ARG
    # NaN in f -> non-finite residual status, never a trap
    import torch
    f = torch.full((9, 9), float("nan"), dtype=torch.float64, device="cuda")
    u = torch.zeros((9, 9), dtype=torch.float64, device="cuda")
    res = g.solve(u, f)
    assert res.status == mg.ERR_NONFINITE
