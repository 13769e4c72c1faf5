"""GPU parity at the benchmark's full size: 4097 x 4097 nodes, wall tanh
stretching (Eq. tanh) with spacing ratio 1000, f ~ N(0, 1) seed 1, tweed
V(1,1) with full weighting -- the launch configuration bench.py times (the
tiled line path on the five finest levels, FP32 cycles with FP64 refinement).

At this size the oracle cannot run every check quickly, so the checks are:
  * one colour pass (Sec. 3), FP64 and FP32, from a seeded random u:
      - nodes of the other colour are untouched (bit-exact);
      - every node of the relaxed colour satisfies its row of Eq. (prob:DP) to
        a backward error of 4096 eps of the row scale -- a property of an
        exact block solve that holds at any size and covers every block, the
        long centre cross included;
      - sampled blocks (corners, L-blocks of many lengths) equal the oracle's
        solve of that block on the same input within c * eps * Skeel
        condition number of the block, computed from the oracle's dense
        assembly of the block;
  * the FP64 solve: per-cycle relative residual history equal to the
    oracle's within 1e-12, measured convergence factor within 1 %;
  * the FP32 + FP64-refinement solve of bench.py: reaches 1e-10 by the GPU
    norm and by the oracle's FP64 residual of the returned u;
  * both solutions against the oracle's: -L is an M-matrix, so
    ||u - u_ref||_inf <= ||L^-1||_inf (||r||_inf + ||r_ref||_inf), with
    ||L^-1||_inf = max w for L w = -1 (w >= 0, maximum principle), w from the
    oracle; the residuals carry their own FP64 evaluation error, 16 eps times
    the largest row scale.
"""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N = 4096
RATIO = 1000.0
EPS = {np.float64: 2.0 ** -53, np.float32: 2.0 ** -24}


@pytest.fixture(scope="module")
def big(oracle_mod):
    c = I.c_for_ratio(N, RATIO, "wall")
    x = I.wall_coords(N, c)
    f = I.rhs_gaussian(N + 1, N + 1, 1)
    P = oracle_mod.Problem(x, x)
    return x, f, P


@pytest.fixture(scope="module")
def grid(mg, big):
    x, _, _ = big
    return mg.Grid(x, x)


@pytest.fixture(scope="module")
def oracle_solution(big):
    """The oracle's FP64 V(1,1) tweed solve to 1e-10 from u = 0, with history."""
    _, f, P = big
    u, hist, _ = P.solve(np.zeros_like(f), f, "tweed", 1, 1, tol=1e-10, max_cycles=40)
    return u, np.asarray(hist)


@pytest.fixture(scope="module")
def linv_norm(big):
    """||L^-1||_inf = max w, L w = -1 on the interior, w = 0 on the boundary."""
    _, f, P = big
    rhs = -np.ones_like(f)
    w, _, _ = P.solve(np.zeros_like(f), rhs, "tweed", 1, 1, tol=1e-8, max_cycles=40)
    return float(np.max(np.abs(w)))


def residual_bound(P, u, f):
    """||f - L u||_inf plus its FP64 evaluation error."""
    r = P.residual(u, f)
    return np.max(np.abs(r[1:-1, 1:-1])) + 16 * EPS[np.float64] * np.max(row_scale(P, u, f))


def row_scale(P, u, f):
    """|f| + sum over the 5-point row of |coefficient * u| (Eq. prob:DP)."""
    W, E, S, N_ = P.coeffs()
    C = (W[None, :] + E[None, :]) + (S[:, None] + N_[:, None])
    s = np.abs(f) + C * np.abs(u)
    s[:, 1:-1] += W[None, 1:-1] * np.abs(u[:, :-2]) + E[None, 1:-1] * np.abs(u[:, 2:])
    s[1:-1, :] += S[1:-1, None] * np.abs(u[:-2, :]) + N_[1:-1, None] * np.abs(u[2:, :])
    return s


def colour_mask(P, colour):
    part = P.partition("tweed")
    owner = P.owner("tweed")
    colours = part[:, 1]
    m = np.zeros(owner.shape, dtype=bool)
    inside = owner >= 0
    m[inside] = colours[owner[inside]] == colour
    return m


def gpu_pass(mg, grid, u_in, f, colour, dtype, path="auto"):
    import torch
    ud = torch.tensor(u_in.astype(dtype), device="cuda")
    fd = torch.tensor(f.astype(dtype), device="cuda")
    dt = "f64" if dtype == np.float64 else "f32"
    grid.set_line_path(0, "tweed", dt, path)
    try:
        grid.colour_pass(ud, fd, "tweed", colour)
    finally:
        grid.set_line_path(0, "tweed", dt, "auto")
    torch.cuda.synchronize()
    return ud.cpu().numpy()


@pytest.mark.parametrize("dtype,path", [(np.float64, "auto"), (np.float32, "auto"), (np.float32, "cluster")],
                         ids=["f64", "f32", "f32-cluster"])
@pytest.mark.parametrize("colour", [0, 1])
def test_fullsize_pass_backward_error(mg, grid, big, dtype, path, colour):
    _, f, P = big
    u_in = I.random_field(N + 1, N + 1, 11 + colour).astype(dtype)
    f_t = f.astype(dtype)
    out = gpu_pass(mg, grid, u_in, f_t, colour, dtype, path)
    mine = colour_mask(P, colour)
    # the other colour and the boundary are not written
    assert np.array_equal(out[~mine], u_in[~mine])
    # the relaxed colour solves its rows.  The tiled path solves each 32-node
    # chunk between end values taken from the reduced system, so the rounding
    # of those ends reaches the chunk's rows amplified by the chunk's
    # condition number, at most ~32^2 for a 32-node line of the 5-point
    # operator: bound (32^2 * 4) eps.  The FP32 pass also carries the FP32
    # rounding of its coefficients (one eps per term of the row scale).  A
    # wrong index or a dropped term gives a backward error of order 1.
    o64, f64 = out.astype(np.float64), f_t.astype(np.float64)
    r = P.residual(o64, f64)
    s = row_scale(P, o64, f64)
    berr = np.max(np.abs(r[mine]) / s[mine])
    assert berr <= 4096 * EPS[dtype], berr


def sample_blocks(P, colour, rng, count=6, max_nodes=1600):
    part = P.partition("tweed")
    idx = np.flatnonzero((part[:, 1] == colour) & (part[:, 2] <= max_nodes))
    sizes = part[idx, 2]
    order = idx[np.argsort(sizes, kind="stable")]
    pick = {int(order[0]), int(order[-1]), int(order[len(order) // 2])}
    pick.update(int(b) for b in rng.choice(idx, size=count, replace=False))
    return sorted(pick)


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_fullsize_pass_sampled_blocks(mg, grid, big, dtype):
    _, f, P = big
    rng = np.random.default_rng(5)
    for colour in (0, 1):
        u_in = I.random_field(N + 1, N + 1, 21 + colour).astype(dtype)
        f_t = f.astype(dtype)
        out = gpu_pass(mg, grid, u_in, f_t, colour, dtype)
        u64, f64 = u_in.astype(np.float64), f_t.astype(np.float64)
        for b in sample_blocks(P, colour, rng):
            nodes = P.block_nodes("tweed", b)
            ii = np.array([p[0] for p in nodes])
            jj = np.array([p[1] for p in nodes])
            ref = P.block_solve("tweed", b, u64.copy(), f64)[jj, ii]
            got = out[jj, ii].astype(np.float64)
            A, _ = P.block_dense("tweed", b, u64, f64)
            # Skeel condition of the block at its solution: || |A^-1| |A| |x| || / ||x||
            # (A is an M-matrix up to sign: A^-1 has one sign, so |A^-1| = |inv(A)|)
            skeel = np.max(np.abs(np.linalg.inv(A)) @ (np.abs(A) @ np.abs(ref))) / np.max(np.abs(ref))
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err <= 64 * EPS[dtype] * max(skeel, 1.0), (colour, b, len(nodes), err, skeel)


def test_fullsize_solve_f64_matches_oracle(mg, grid, big, oracle_solution, linv_norm):
    import torch
    _, f, P = big
    u_ref, hist_ref = oracle_solution
    ud = torch.zeros((N + 1, N + 1), dtype=torch.float64, device="cuda")
    res = grid.solve(ud, torch.tensor(f, device="cuda"), smoother="tweed", nu1=1, nu2=1, tol=1e-10,
                     max_cycles=40)
    assert res.status == mg.OK
    k = min(len(res.history), len(hist_ref))
    assert len(res.history) == len(hist_ref)
    assert np.abs(res.history[:k] - hist_ref[:k]).max() <= 1e-12
    cf_gpu = (res.history[k - 1] / res.history[0]) ** (1.0 / (k - 1))
    cf_ref = (hist_ref[k - 1] / hist_ref[0]) ** (1.0 / (k - 1))
    assert abs(cf_gpu - cf_ref) <= 0.01 * cf_ref
    u = ud.cpu().numpy()
    bound = 1.01 * linv_norm * (residual_bound(P, u, f) + residual_bound(P, u_ref, f))
    assert np.max(np.abs(u - u_ref)) <= bound, (np.max(np.abs(u - u_ref)), bound)


def test_fullsize_solve_f32_refine(mg, grid, big, oracle_solution, linv_norm):
    """The configuration bench.py times, parameter for parameter (bench.HEADLINE:
    V(1,1), 3 FP32 cycles per refinement step, every level down to the FP64
    coarsest solve)."""
    import torch
    from bench import HEADLINE
    _, f, P = big
    u_ref, _ = oracle_solution
    ud = torch.zeros((N + 1, N + 1), dtype=torch.float64, device="cuda")
    res = grid.solve(ud, torch.tensor(f, device="cuda"), **HEADLINE)
    assert res.status == mg.OK and res.rel_res <= 1e-10
    u = ud.cpu().numpy()
    r = P.residual(u, f)
    rel = np.sqrt(np.sum(r[1:-1, 1:-1] ** 2)) / np.sqrt(np.sum(f[1:-1, 1:-1] ** 2))
    assert rel <= 1e-10, rel
    bound = 1.01 * linv_norm * (residual_bound(P, u, f) + residual_bound(P, u_ref, f))
    err = np.max(np.abs(u - u_ref))
    assert err <= bound, (err, bound)
