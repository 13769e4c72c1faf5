"""Gradients through the solve (torch.autograd.Function over mg_solve /
mg_solve_adjoint / mg_boundary_adjoint) against
  * the oracle's gradient (dense transpose solve, itself pinned by central
    differences) on a small stretched grid, FP64 and FP32 + FP64 refinement;
  * central differences of the quadratic loss 0.5 ||u - u_target||^2 on the
    2049 x 2049 wall-clustered grid (spacing ratio 500), u_target ~ N(0,1)
    seed 3, 64 directions ~ N(0,1) (normalised) seed 4 for f and 16 for the
    boundary data, FP32 + refinement.  The loss is quadratic in f and g, so
    central differences are exact up to the solve tolerance and rounding.
"""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup_small(mg, oracle_mod):
    x = I.wall_coords(48, 2.0)
    y = I.centre_coords(40, 1.2)
    P = oracle_mod.Problem(x, y)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(P.shape())
    g = rng.standard_normal(P.shape())
    ut = rng.standard_normal(P.shape())
    return mg.Grid(x, y), P, f, g, ut


# solves to a relative residual of 1e-11 (the FP64 rounding floor of this grid
# with O(1) boundary data is near 5e-12); the gradient error is that residual
# amplified by the conditioning of A (below 1e4 here): bound 1e-7
@pytest.mark.parametrize("precision,tol,bound", [("f64", 1e-11, 1e-7), ("f32_refine", 1e-11, 1e-7)])
def test_autograd_matches_oracle_gradient(mg, oracle_mod, precision, tol, bound):
    import torch
    from paper_2110_08389_gb300.autograd import tweed_solve
    grid, P, f, g, ut = _setup_small(mg, oracle_mod)
    loss_ref, u_ref, gf_ref, gg_ref = oracle_mod.quadratic_loss_gradient(P, f, g, ut)
    fd = torch.tensor(f, device="cuda", requires_grad=True)
    gd = torch.tensor(g, device="cuda", requires_grad=True)
    u = tweed_solve(grid, fd, gd, precision=precision, tol=tol)
    loss = 0.5 * ((u - torch.tensor(ut, device="cuda")) ** 2).sum()
    loss.backward()
    assert float(loss) == pytest.approx(loss_ref, rel=1e-9)
    gf, gg = fd.grad.cpu().numpy(), gd.grad.cpu().numpy()
    ef = np.max(np.abs(gf - gf_ref)) / np.max(np.abs(gf_ref))
    eg = np.max(np.abs(gg - gg_ref)) / np.max(np.abs(gg_ref))
    assert ef <= bound and eg <= bound, (ef, eg)


def test_config4_finite_differences(mg):
    import torch
    from paper_2110_08389_gb300.autograd import tweed_solve
    n = 2048
    x = I.wall_coords(n, I.c_for_ratio(n, 500.0))
    grid = mg.Grid(x, x)
    f = torch.tensor(I.rhs_gaussian(n + 1, n + 1, 3), device="cuda")
    ut = torch.tensor(np.random.Generator(np.random.PCG64(3)).standard_normal((n + 1, n + 1))[::-1].copy(),
                      device="cuda")
    g = torch.zeros_like(f)
    kw = dict(precision="f32_refine", tol=1e-11)
    fr = f.clone().requires_grad_(True)
    gr = g.clone().requires_grad_(True)
    u = tweed_solve(grid, fr, gr, **kw)
    (0.5 * ((u - ut) ** 2).sum()).backward()
    gf, gg = fr.grad.detach(), gr.grad.detach()

    def loss(ff, gg_):
        with torch.no_grad():
            uu = tweed_solve(grid, ff, gg_, **kw)
            return 0.5 * float(((uu - ut) ** 2).sum())

    rng = np.random.Generator(np.random.PCG64(4))
    inner = torch.zeros_like(f, dtype=torch.bool)
    inner[1:-1, 1:-1] = True
    h = float(f.norm())  # the loss is quadratic: any step gives the exact central difference
    got, want = [], []
    for s in range(64):
        d = torch.tensor(rng.standard_normal((n + 1, n + 1)), device="cuda")
        d = torch.where(inner, d, torch.zeros_like(d))
        d /= d.norm()
        got.append((loss(f + h * d, g) - loss(f - h * d, g)) / (2 * h))
        want.append(float((gf * d).sum()))
    got, want = np.array(got), np.array(want)
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want)), (got[:4], want[:4])
    got, want = [], []
    for s in range(16):
        d = torch.tensor(rng.standard_normal((n + 1, n + 1)), device="cuda")
        d = torch.where(inner, torch.zeros_like(d), d)
        d /= d.norm()
        got.append((loss(f, g + d) - loss(f, g - d)) / 2.0)
        want.append(float((gg * d).sum()))
    got, want = np.array(got), np.array(want)
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want)), (got[:4], want[:4])
