"""The refinement step of the FP32+refine solve (Sec. 4 step (6) on the FP64
iterate): the update u + e and the next FP64 residual run as one kernel,
which writes the new iterate into a second array, so that the iterate
alternates between the caller's u and the grid's own copy from step to step.

After 1, 2, 3 and 4 refinement steps (an unreachable tolerance stops the
solve on the step cap, so odd counts end in the grid's copy and must come
back) the returned u must keep its Dirichlet data bit for bit, and the
relative residual the solver reported must be the oracle's FP64 residual of
the returned u: a step that updated the wrong array, lost the boundary of
the second array or skipped the copy back fails it.  The same holds for a
packed batch, whose members must also equal their single solves bit for
bit."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def cuda(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def oracle_rel(P, u, f):
    interior = np.zeros_like(u)
    interior[0, :], interior[-1, :], interior[:, 0], interior[:, -1] = u[0, :], u[-1, :], u[:, 0], u[:, -1]
    r = P.residual(u, f)[1:-1, 1:-1]
    r0 = P.residual(interior, f)[1:-1, 1:-1]
    return np.linalg.norm(r) / np.linalg.norm(r0)


def problem(nx, ny, seed):
    x, y = I.wall_coords(nx, 2.0), I.wall_coords(ny, 2.5)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((ny + 1, nx + 1))
    f = rng.standard_normal((ny + 1, nx + 1))
    return x, y, g, f


@pytest.mark.parametrize("guess", [0, 1], ids=["zeroed", "caller"])
@pytest.mark.parametrize("steps", [1, 2, 3, 4])
def test_refinement_iterate_and_residual_after_each_step(mg, oracle_mod, steps, guess):
    """guess 0: the solver zeroes the interior and its first residual comes
    with the scale norm (f - B g); guess 1: the caller's u is the first
    iterate and its residual is a separate FP64 defect."""
    x, y, gdat, f = problem(192, 136, 31)
    P = oracle_mod.Problem(x, y)
    grid = mg.Grid(x, y)
    if guess:
        gdat = gdat.copy()
        gdat[1:-1, 1:-1] = np.random.default_rng(32).standard_normal((gdat.shape[0] - 2, gdat.shape[1] - 2))
    ud = cuda(gdat)
    res = grid.solve(ud, cuda(f), smoother="tweed", nu1=1, nu2=1, precision="f32_refine", tol=1e-30, early_stop=0,
                     inner_cycles=2, max_outer=steps, max_cycles=1000, use_initial_guess=guess)
    assert res.status == mg.ERR_NOT_CONVERGED and res.outer_iters == steps
    u = ud.cpu().numpy()
    for a, b in ((u[0, :], gdat[0, :]), (u[-1, :], gdat[-1, :]), (u[:, 0], gdat[:, 0]), (u[:, -1], gdat[:, -1])):
        assert np.array_equal(a, b)
    want = oracle_rel(P, u, f)
    assert abs(res.rel_res - want) <= 1e-9 * want, (res.rel_res, want)
    assert res.rel_res < 0.1 * res.history[0]  # the steps made progress


def test_packed_batch_iterates_match_single_solves(mg, oracle_mod):
    import torch
    probs = [problem(128, 128, 40 + k) for k in range(3)]
    grids = [mg.Grid(x, y) for x, y, _, _ in probs]
    kw = dict(smoother="tweed", nu1=1, nu2=1, precision="f32_refine", tol=1e-30, early_stop=0, inner_cycles=2, max_outer=3,
              max_cycles=1000)
    us = [cuda(gd) for _, _, gd, _ in probs]
    fs = [cuda(f) for _, _, _, f in probs]
    n0 = mg.kernel_launches()
    out = mg.Batch(grids).solve(us, fs, **kw)
    n_batch = mg.kernel_launches() - n0
    n0 = mg.kernel_launches()
    singles = []
    for (x, y, gdat, f), g in zip(probs, grids):
        ud = cuda(gdat)
        singles.append((ud, g.solve(ud, cuda(f), **kw)))
    n_single = mg.kernel_launches() - n0
    torch.cuda.synchronize()
    assert n_batch < 0.75 * n_single  # the three members ran as one packed group
    for (x, y, gdat, f), ub, r, (ud, single) in zip(probs, us, out, singles):
        assert r.status == mg.ERR_NOT_CONVERGED and r.outer_iters == 3
        assert np.array_equal(ub.cpu().numpy(), ud.cpu().numpy())
        assert single.rel_res == r.rel_res
        P = oracle_mod.Problem(x, y)
        want = oracle_rel(P, ub.cpu().numpy(), f)
        assert abs(r.rel_res - want) <= 1e-9 * want
