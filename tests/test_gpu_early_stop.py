"""mg_params.early_stop: a solve that converges gives bit for bit the same
result with it; one that cannot reach the tolerance within its caps stops
as soon as the last step's reduction shows it (from the third step on), with
the history so far equal to the full run's; batches give what single solves
give."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _grid(mg, n, kind, c=None, ratio=None):
    x = I.coords(n, kind, c=c) if c is not None else I.coords(n, kind, ratio=ratio)
    return mg.Grid(x, x)


def _rhs(n, seed):
    import torch
    return torch.tensor(I.rhs_gaussian(n + 1, n + 1, seed), device="cuda")


@pytest.mark.parametrize("precision", ["f64", "f32_refine"])
def test_converging_solve_unchanged(mg, precision):
    import torch
    g = _grid(mg, 256, "wall", ratio=300.0)
    f = _rhs(256, 3)
    kw = dict(smoother="tweed", nu1=1, nu2=1, tol=1e-10, precision=precision, max_cycles=100, max_outer=20)
    u0 = torch.zeros_like(f)
    u1 = torch.zeros_like(f)
    r0 = g.solve(u0, f, **kw)
    r1 = g.solve(u1, f, early_stop=1, **kw)
    assert r0.status == r1.status == mg.OK
    assert (r0.cycles, r0.outer_iters) == (r1.cycles, r1.outer_iters)
    assert np.array_equal(r0.history, r1.history)
    assert torch.equal(u0, u1)


@pytest.mark.parametrize("precision", ["f64", "f32_refine"])
def test_hopeless_solve_stops_early(mg, precision):
    """Wireframe under strong wall clustering (c = 3) does not converge
    (Sec. 6): with early_stop the solve gives up after a few steps."""
    import torch
    g = _grid(mg, 128, "wall", c=3.0)
    f = _rhs(128, 4)
    kw = dict(smoother="wireframe", nu1=1, nu2=1, tol=1e-10, precision=precision, max_cycles=60, max_outer=20)
    u0 = torch.zeros_like(f)
    r0 = g.solve(u0, f, **kw)
    u1 = torch.zeros_like(f)
    r1 = g.solve(u1, f, early_stop=1, **kw)
    assert r0.status == r1.status == mg.ERR_NOT_CONVERGED
    steps0 = len(r0.history) - 1
    steps1 = len(r1.history) - 1
    assert 3 <= steps1 < steps0, (steps0, steps1)
    assert np.array_equal(r1.history, r0.history[: steps1 + 1])
    # the stop was justified: at the last step's rate the steps left fall short
    rate = r1.history[-1] / r1.history[-2]
    assert rate >= 1.0 or r1.history[-1] * rate ** (steps0 - steps1) > 1e-10


def test_early_stop_in_a_batch_equals_single_solves(mg):
    import torch
    grids = [_grid(mg, 128, "wall", c=3.0), _grid(mg, 128, "wall", ratio=100.0), _grid(mg, 64, "wall", c=3.0)]
    fs = [_rhs(128, 5), _rhs(128, 6), _rhs(64, 7)]
    kws = [dict(smoother="wireframe", nu1=1, nu2=1, tol=1e-10, precision="f32_refine", max_cycles=60, max_outer=20,
                early_stop=1),
           dict(smoother="tweed", nu1=1, nu2=1, tol=1e-10, precision="f32_refine", max_cycles=60, max_outer=20,
                early_stop=1),
           dict(smoother="wireframe", nu1=1, nu2=1, tol=1e-10, precision="f64", max_cycles=60, early_stop=1)]
    us = [torch.zeros_like(f) for f in fs]
    res = mg.Batch(grids).solve(us, fs, [mg.default_params(**kw) for kw in kws])
    torch.cuda.synchronize()
    for k in range(3):
        u1 = torch.zeros_like(fs[k])
        r1 = grids[k].solve(u1, fs[k], **kws[k])
        assert res[k].status == r1.status, k
        assert np.array_equal(res[k].history, r1.history), k
        assert torch.equal(us[k], u1), k
