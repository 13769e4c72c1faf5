"""Pins of the CPU oracle against what the paper and the mathematics fix:
closed forms of the operator, the block counts / shapes / flop totals printed
in Sec. 3, the worked block systems of Sec. 3, complementarity (Sec. 8),
block solves against dense LU, multigrid against a dense direct solve, O(h^2)
convergence to a manufactured solution, transfer duality (Sec. 4) and the
qualitative convergence claims of Sec. 6."""
import math

import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I


def _prob(oracle_mod, nx, ny=None, kind="uniform", c=0.0):
    ny = nx if ny is None else ny
    f = {"uniform": lambda n: I.uniform_coords(n), "wall": lambda n: I.wall_coords(n, c),
         "centre": lambda n: I.centre_coords(n, c)}[kind]
    return oracle_mod.Problem(f(nx), f(ny))


# ------------------------------------------------------------------ operator

def test_uniform_coefficients(oracle_mod):
    """Sec. 2: on an unstretched grid W = E = 1/dx^2 and S = N = 1/dy^2."""
    P = oracle_mod.Problem(I.uniform_coords(8), np.linspace(0, 2.0, 13))
    W, E, S, N = P.coeffs()
    assert np.allclose(W[1:-1], 64.0) and np.allclose(E[1:-1], 64.0)
    assert np.allclose(S[1:-1], 36.0) and np.allclose(N[1:-1], 36.0)


@pytest.mark.parametrize("kind,c", [("wall", 3.0), ("centre", 1.5)])
def test_operator_exact_on_quadratics(oracle_mod, kind, c):
    """The three-point formula of Sec. 2 is exact for polynomials of degree 2 on
    any grid: L(1) = 0, L(x) = L(y) = 0 and L(x^2 + y^2) = 4 at every interior
    node (boundary values included)."""
    P = _prob(oracle_mod, 24, 18, kind, c)
    X, Y = np.meshgrid(P.x, P.y)
    for u, val in [(np.ones_like(X), 0.0), (X, 0.0), (3 * Y - 1, 0.0), (X ** 2 + Y ** 2, 4.0)]:
        out = P.apply(u)
        assert np.allclose(out[1:-1, 1:-1], val, atol=1e-8 * np.abs(out).max() + 1e-8)


def test_symmetric_scaled_operator(oracle_mod):
    """D L is symmetric on the interior with D = diag(dx_i dy_j)."""
    P = _prob(oracle_mod, 10, 8, "wall", 2.5)
    ny1, nx1 = P.shape()
    n = (ny1 - 2) * (nx1 - 2)
    cols = []
    for k in range(n):
        e = np.zeros((ny1, nx1))
        e[1:-1, 1:-1].flat[k] = 1.0
        cols.append(P.apply(e)[1:-1, 1:-1].ravel())
    L = np.stack(cols, axis=1)
    dx = 0.5 * (P.x[2:] - P.x[:-2])
    dy = 0.5 * (P.y[2:] - P.y[:-2])
    D = np.outer(dy, dx).ravel()
    DL = D[:, None] * L
    assert np.allclose(DL, DL.T, rtol=1e-12, atol=1e-12 * np.abs(DL).max())
    assert not np.allclose(L, L.T)  # L itself is not symmetric on a stretched grid


# ---------------------------------------------------------------- partitions

def _counts(info):
    types, legs = info[:, 0], info[:, 3]
    return {"point": int((types == 0).sum()), "path": int((types == 1).sum()),
            "cycle": int((types == 2).sum()), "star3": int(((types == 3) & (legs == 3)).sum()),
            "star4": int(((types == 3) & (legs == 4)).sum())}


@pytest.mark.parametrize("n", [7, 15, 31, 63])
def test_tweed_square_counts(oracle_mod, n):
    """Sec. 3: 4 corner points, 2(n-3) two-legged blocks, one four-legged
    centre cross (n = interior nodes per side)."""
    P = _prob(oracle_mod, n + 1)
    c = _counts(P.partition("tweed"))
    assert c == {"point": 4, "path": 2 * (n - 3), "cycle": 0, "star3": 0, "star4": 1}


@pytest.mark.parametrize("n", [7, 15, 31, 63])
def test_wireframe_square_counts(oracle_mod, n):
    """Sec. 3: (n-1)/2 concentric rings of 8i nodes plus the centre point."""
    P = _prob(oracle_mod, n + 1)
    info = P.partition("wireframe")
    c = _counts(info)
    assert c == {"point": 1, "path": 0, "cycle": (n - 1) // 2, "star3": 0, "star4": 0}
    sizes = sorted(int(s) for t, _, s, _ in info if t == 2)
    assert sizes == [8 * i for i in range(1, (n - 1) // 2 + 1)]


@pytest.mark.parametrize("nx,ny", [(16, 8), (32, 16), (24, 8)])
def test_rectangular_shapes(oracle_mod, nx, ny):
    """Sec. 3: nx > ny gives two three-legged tweed blocks plus straight lines,
    and wireframe rings ending in one x-line."""
    P = _prob(oracle_mod, nx, ny)
    c = _counts(P.partition("tweed"))
    assert c["star3"] == 2 and c["star4"] == 0 and c["point"] == 4
    w = P.partition("wireframe")
    cw = _counts(w)
    assert cw["cycle"] == ny // 2 - 1 and cw["path"] == 1 and cw["point"] == 0
    line = [s for t, _, s, _ in w if t == 1][0]
    assert line == nx - ny + 1


@pytest.mark.parametrize("n", [7, 15, 63, 127])
def test_flop_totals(oracle_mod, n):
    """The printed totals 12n^2 - 10n + 11 (tweed) and 18n^2 - 8n - 1
    (wireframe) follow from the oracle's block shapes and the paper's
    per-block costs: pointwise relaxation 9; an m-legged block with legs of p
    nodes 8mp + m + 1 plus 4 per right-hand-side node (the paper counts the
    branch point's RHS for the two-legged blocks but not for the centre
    cross); a ring of s nodes 14s - 16 plus 4 per node."""
    P = _prob(oracle_mod, n + 1)
    tw = 0
    for t, _, size, legs in P.partition("tweed"):
        if t == 0:
            tw += 9
        elif t == 1:                    # two legs of p nodes meeting at a corner
            p = (size - 1) // 2
            tw += 4 * size + 8 * 2 * p + 2 + 1
        else:                           # centre cross
            p = (size - 1) // legs
            tw += 4 * (size - 1) + 8 * legs * p + legs + 1
    assert tw == 12 * n * n - 10 * n + 11
    wf = 0
    for t, _, size, _ in P.partition("wireframe"):
        wf += 9 if t == 0 else 4 * size + 14 * size - 16
    assert wf == 18 * n * n - 8 * n - 1


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 16), (16, 10), (12, 20)])
def test_complementarity_and_decoupling(oracle_mod, nx, ny):
    """Sec. 8: the tweed and wireframe motifs use disjoint sets of grid edges
    whose union is every edge between interior nodes.  Sec. 3: blocks of the
    same colour never share an edge (red-black decoupling)."""
    P = _prob(oracle_mod, nx, ny)
    edges = {}
    for sm in ("tweed", "wireframe"):
        own = P.owner(sm)
        info = P.partition(sm)
        used = set()
        for j in range(1, ny):
            for i in range(1, nx):
                for di, dj in ((1, 0), (0, 1)):
                    a, b = (i, j), (i + di, j + dj)
                    if b[0] >= nx or b[1] >= ny:
                        continue
                    ba, bb = own[a[1], a[0]], own[b[1], b[0]]
                    if ba == bb:
                        used.add((a, b))
                    else:
                        assert info[ba, 1] != info[bb, 1], (sm, a, b)  # different blocks: other colour
        edges[sm] = used
    all_edges = {((i, j), (i + di, j + dj)) for j in range(1, ny) for i in range(1, nx)
                 for di, dj in ((1, 0), (0, 1)) if i + di < nx and j + dj < ny}
    assert edges["tweed"].isdisjoint(edges["wireframe"])
    assert edges["tweed"] | edges["wireframe"] == all_edges


# ------------------------------------------------------- worked block systems

def test_worked_tweed_block(oracle_mod):
    """Sec. 3 worked example: the red block joining at the (4,4) node (1-based;
    (3,3) 0-based) on a uniform grid: legs (2,4),(3,4) and (4,2),(4,3), rows
    EW-C-EW / NS-C-NS, branch row EW, NS, C; the right-hand side of the branch
    row is f - u_{5,4}/dx^2 - u_{4,5}/dy^2 (the printed '+' is a sign typo)."""
    x = I.uniform_coords(8)
    y = np.linspace(0.0, 1.5, 9)
    P = oracle_mod.Problem(x, y)
    dx2, dy2 = (x[1] - x[0]) ** 2, (y[1] - y[0]) ** 2
    own = P.owner("tweed")
    b = own[3, 3]
    nodes = P.block_nodes("tweed", b)
    assert sorted(nodes) == sorted([(1, 3), (2, 3), (3, 3), (3, 1), (3, 2)])
    rng = np.random.default_rng(3)
    u = rng.standard_normal((9, 9))
    f = rng.standard_normal((9, 9))
    A, r = P.block_dense("tweed", b, u, f)
    idx = {nd: k for k, nd in enumerate(nodes)}
    C = -2 / dx2 - 2 / dy2
    assert np.allclose(np.diag(A), C)
    assert A[idx[(2, 3)], idx[(1, 3)]] == pytest.approx(1 / dx2)
    assert A[idx[(2, 3)], idx[(3, 3)]] == pytest.approx(1 / dx2)
    assert A[idx[(3, 2)], idx[(3, 1)]] == pytest.approx(1 / dy2)
    assert A[idx[(3, 3)], idx[(2, 3)]] == pytest.approx(1 / dx2)
    assert A[idx[(3, 3)], idx[(3, 2)]] == pytest.approx(1 / dy2)
    # leg RHS: f_{2,4} - (u_{2,3} + u_{2,5})/dy^2 and the wall value g_{1,4}/dx^2
    k = idx[(1, 3)]
    assert r[k] == pytest.approx(f[3, 1] - (u[2, 1] + u[4, 1]) / dy2 - u[3, 0] / dx2)
    k = idx[(3, 1)]
    assert r[k] == pytest.approx(f[1, 3] - (u[1, 2] + u[1, 4]) / dx2 - u[0, 3] / dy2)
    k = idx[(3, 3)]
    assert r[k] == pytest.approx(f[3, 3] - u[3, 4] / dx2 - u[4, 3] / dy2)


def test_worked_wireframe_ring(oracle_mod):
    """Sec. 3 worked example: the red ring of the 5x5 grid, corners (2,2),
    (2,4), (4,2), (4,4) (1-based): an 8x8 circulant tridiagonal system whose
    couplings alternate EW / NS around the box."""
    x = I.uniform_coords(4)
    y = np.linspace(0.0, 0.5, 5)
    P = oracle_mod.Problem(x, y)
    dx2, dy2 = (x[1] - x[0]) ** 2, (y[1] - y[0]) ** 2
    own = P.owner("wireframe")
    b = own[1, 1]
    nodes = P.block_nodes("wireframe", b)
    ring = [(1, 1), (2, 1), (3, 1), (3, 2), (3, 3), (2, 3), (1, 3), (1, 2)]  # paper's order, 0-based
    assert sorted(nodes) == sorted(ring)
    rng = np.random.default_rng(5)
    u, f = rng.standard_normal((5, 5)), rng.standard_normal((5, 5))
    A, r = P.block_dense("wireframe", b, u, f)
    perm = [nodes.index(p) for p in ring]
    A = A[np.ix_(perm, perm)]
    r = r[perm]
    EW, NS, C = 1 / dx2, 1 / dy2, -2 / dx2 - 2 / dy2
    expect = np.diag([C] * 8)
    pairs = [(0, 1, EW), (1, 2, EW), (2, 3, NS), (3, 4, NS), (4, 5, EW), (5, 6, EW), (6, 7, NS), (7, 0, NS)]
    for a, c, v in pairs:
        expect[a, c] = expect[c, a] = v
    assert np.allclose(A, expect)
    # first row: f_{2,2} - u_{1,2}/dx^2 - u_{2,1}/dy^2 (1-based)
    assert r[0] == pytest.approx(f[1, 1] - u[1, 0] / dx2 - u[0, 1] / dy2)
    # fourth row: f_{4,3} - u_{3,3}/dx^2 - u_{5,3}/dx^2 (centre node is black)
    assert r[3] == pytest.approx(f[2, 3] - u[2, 2] / dx2 - u[2, 4] / dx2)


# ------------------------------------------------------------ block solvers

@pytest.mark.parametrize("smoother", ["checkerboard", "zebra_x", "zebra_y", "tweed", "wireframe"])
@pytest.mark.parametrize("nx,ny,kind,c", [(16, 16, "wall", 2.0), (20, 12, "centre", 1.5), (12, 18, "wall", 1.0)])
def test_block_solves_match_dense_lu(oracle_mod, smoother, nx, ny, kind, c):
    """Thomas, m-legged Thomas (Eq. mLThomas) and circulant Thomas (Eq.
    CircTri) against Gaussian elimination on the assembled block."""
    P = _prob(oracle_mod, nx, ny, kind, c)
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    info = P.partition(smoother)
    worst = 0.0
    for b in range(len(info)):
        nodes = P.block_nodes(smoother, b)
        A, r = P.block_dense(smoother, b, u0, f)
        x = oracle_mod.dense_solve(A, r)
        u = u0.copy()
        P.block_solve(smoother, b, u, f)
        got = np.array([u[j, i] for i, j in nodes])
        worst = max(worst, np.abs(got - x).max() / (np.abs(x).max() + 1e-300))
    assert worst < 1e-12


@pytest.mark.parametrize("smoother", ["checkerboard", "zebra_x", "zebra_y", "tweed", "wireframe"])
def test_relaxed_rows_have_zero_residual(oracle_mod, smoother):
    """After a colour pass every row of that colour is satisfied exactly (up
    to rounding) with the other colour held fixed."""
    P = _prob(oracle_mod, 40, 32, "wall", 3.0)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    own = P.owner(smoother)
    col = P.partition(smoother)[:, 1]
    W, E, S, N = P.coeffs()
    for colour in (0, 1):
        P.colour_pass(u, f, smoother, colour)
        d = P.residual(u, f)
        scale = (np.abs(W)[None, :] + np.abs(E)[None, :] + np.abs(S)[:, None] + np.abs(N)[:, None]) * np.abs(u).max()
        mask = np.zeros_like(u, dtype=bool)
        mask[1:-1, 1:-1] = col[own[1:-1, 1:-1]] == colour
        assert np.abs(d[mask] / scale[mask]).max() < 1e-13


# ---------------------------------------------------------------- multigrid

@pytest.mark.parametrize("smoother", ["checkerboard", "alt_zebra", "tweed", "wireframe", "alt_tw"])
@pytest.mark.parametrize("nx,ny", [(8, 8), (6, 8), (4, 2)])
def test_multigrid_equals_dense_lu(oracle_mod, smoother, nx, ny):
    """On grids of at most 9x9 nodes the multigrid iteration converges to the
    dense-LU solution of Eq. (prob:DP), boundary data included."""
    P = oracle_mod.Problem(I.wall_coords(nx, 1.5), I.wall_coords(ny, 1.5))
    rng = np.random.default_rng(7)
    g = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    ref = P.direct_solve(g, f)
    u, hist, _ = P.solve(g, f, smoother, 1, 1, tol=1e-13, max_cycles=200)
    assert hist[-1] <= 1e-13
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()


def test_manufactured_second_order(oracle_mod):
    """O(h^2): with u* = sin(pi x) sin(pi y) the discretisation error of the
    solved system drops by ~4 per halving of h on a fixed stretching."""
    errs = []
    for n in (16, 32, 64, 128):
        x = I.wall_coords(n, 2.0)
        P = oracle_mod.Problem(x, x)
        ue, f = I.manufactured(x, x)
        u, hist, _ = P.solve(np.zeros_like(f), f, "tweed", 2, 2, tol=1e-12)
        errs.append(np.abs(u - ue).max())
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios


def test_fw_is_quarter_transpose_of_bilinear(oracle_mod):
    """Sec. 4: bilinear interpolation is the dual of full weighting,
    <R d, v>_coarse = 1/4 <d, P v>_fine for zero-boundary d, v."""
    P = oracle_mod.Problem(I.wall_coords(16, 2.0), I.uniform_coords(12))
    rng = np.random.default_rng(4)
    d = I.random_field(*P.shape(0), seed=8)
    v = I.random_field(*P.shape(1), seed=9)
    Rd = P.restrict(d, oracle_mod.FW)
    Pv = P.prolong_add(v, np.zeros(P.shape(0)))
    assert np.sum(Rd * v) == pytest.approx(0.25 * np.sum(d * Pv), rel=1e-13)
    # prolongation reproduces coarse values at coinciding nodes and is linear
    assert np.allclose(Pv[::2, ::2], v)
    del rng


def test_tweed_converges_where_point_and_wall_parallel_smoothers_fail(oracle_mod):
    """Sec. 6 (Fig. 9, c = 3): tweed converges fast under near-wall stretching
    while checkerboard and wireframe stall; Sec. 6 (Fig. 10): wireframe is the
    fast one under near-centre stretching."""
    x = I.wall_coords(64, 3.0)
    P = oracle_mod.Problem(x, x)
    f = I.rhs_uniform(65, 65, seed=0)
    rates = {}
    for sm in ("tweed", "checkerboard", "wireframe", "alt_zebra"):
        _, hist, _ = P.solve(np.zeros_like(f), f, sm, 1, 1, tol=1e-30, max_cycles=8)
        rates[sm] = (hist[-1] / hist[0]) ** (1 / 8)
    assert rates["tweed"] < 0.15 and rates["alt_zebra"] < 0.15
    assert rates["checkerboard"] > 0.7 and rates["wireframe"] > 0.7
    xc = I.centre_coords(64, 1.5)
    Pc = oracle_mod.Problem(xc, xc)
    rc = {}
    for sm in ("wireframe", "tweed"):
        _, hist, _ = Pc.solve(np.zeros_like(f), f, sm, 1, 1, tol=1e-30, max_cycles=8)
        rc[sm] = (hist[-1] / hist[0]) ** (1 / 8)
    assert rc["wireframe"] < 0.15 and rc["tweed"] > 0.5


def test_solve_history_shape(oracle_mod):
    x = I.wall_coords(64, I.c_for_ratio(64, 100.0))
    P = oracle_mod.Problem(x, x)
    ue, f = I.manufactured(x, x, noise=1e-3, seed=0)
    u, hist, hmax = P.solve(np.zeros_like(f), f, "tweed", 2, 2, tol=1e-10)
    assert hist[0] == pytest.approx(1.0)
    assert hist[-1] <= 1e-10 and len(hist) < 15
    assert np.all(np.diff(np.log(hist)) < 0)


def test_stretching_maps():
    """Eq. (tanh): c = 1.5 and c = 3.0 at 128 intervals give spacing ratios 5.42
    and 96.6; Eq. (tanh_inv) clusters at the centre; both are symmetric."""
    assert I.spacing_ratio(I.wall_coords(128, 1.5)) == pytest.approx(5.4165, abs=1e-3)
    assert I.spacing_ratio(I.wall_coords(128, 3.0)) == pytest.approx(96.63, abs=1e-2)
    x = I.centre_coords(64, 1.5)
    d = np.diff(x)
    assert d[31] < d[0] and np.allclose(x + x[::-1], 1.0)
    assert I.c_for_ratio(4096, 1000.0) == pytest.approx(4.147788, abs=1e-5)


# ------------------------------------------------------------------ W-cycle
# Sec. 4 names the W-cycle only among "other cycling strategies"; these pins
# come from the mathematics of the cycle (gamma = 2 coarse visits per level).

def test_w_cycle_equals_v_cycle_on_two_levels(oracle_mod):
    """With two levels the coarse level is solved exactly, so the second
    coarse visit sees a zero defect and changes nothing: one W-cycle equals
    one V-cycle bit for bit.  Catches a second visit that adds its correction
    again or starts from a stale coarse right-hand side."""
    P = _prob(oracle_mod, 16, 12, "wall", 2.0)
    assert P.nlev == 2
    rng = np.random.default_rng(21)
    g = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    for sm in ("checkerboard", "tweed", "alt_tw"):
        uv, uw = g.copy(), g.copy()
        for _ in range(3):
            P.cycle(uv, f, sm, 1, 1, gamma=1)
            P.cycle(uw, f, sm, 1, 1, gamma=2)
        assert np.array_equal(uv, uw), sm


@pytest.mark.parametrize("smoother", ["checkerboard", "tweed", "alt_zebra"])
def test_w_cycle_converges_to_dense_lu(oracle_mod, smoother):
    """On a three-level stretched grid the W(1,1) iteration converges to the
    dense-LU solution of Eq. (prob:DP), boundary data included.  Catches a
    W-cycle whose coarse visits leave a wrong fixed point (a dropped or
    doubled correction, a transposed transfer)."""
    P = _prob(oracle_mod, 32, 24, "wall", 2.0)
    assert P.nlev == 3
    rng = np.random.default_rng(22)
    g = rng.standard_normal(P.shape())
    f = rng.standard_normal(P.shape())
    ref = P.direct_solve(g, f)
    u, hist, _ = P.solve(g, f, smoother, 1, 1, gamma=2, tol=1e-13, max_cycles=200)
    assert hist[-1] <= 1e-13
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("smoother,rho", [("checkerboard", 0.0739), ("alt_zebra", 0.0391), ("tweed", 0.0621)])
def test_w_cycle_factor_matches_two_grid_radius(oracle_mod, smoother, rho):
    """A W-cycle solves each coarse problem almost exactly (two visits, each
    reducing the coarse error by the cycle's own small factor), so on four
    levels its asymptotic factor is the two-grid spectral radius of Sec. 5.
    Table 1 (uniform grid, full weighting, nu = nu1 + nu2 = 2): checkerboard
    .0739, alternating zebra .0391, tweed .0621 (R7: 64 intervals).  The
    factor is the last-cycle residual ratio after 30 renormalised W(1,1)
    cycles from a random error with f = 0.  A W-cycle that restarts its
    second coarse visit from zero is a V-cycle, whose factor here is .115 for
    checkerboard and .053 for alternating zebra, and fails this pin."""
    P = _prob(oracle_mod, 64)
    assert P.nlev == 4
    u = I.random_field(65, 65, seed=23)
    f = np.zeros_like(u)
    ratio = None
    for _ in range(30):
        r0 = np.linalg.norm(P.residual(u, f)[1:-1, 1:-1])
        u /= r0
        P.cycle(u, f, smoother, 1, 1, gamma=2)
        ratio = np.linalg.norm(P.residual(u, f)[1:-1, 1:-1])
    assert abs(ratio / rho - 1.0) <= 0.03, (smoother, ratio, rho)
