"""mg_batch_solve: many independent problems (sizes, stretchings, boundary
data all different) solved together must give, problem by problem, exactly
what mg_solve gives for the problem alone -- the same kernels and captured
cycle sequences run on other streams, only the host waits are shared."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PROBLEMS = [  # (nx, ny, kind, ratio); centre clustering kept mild, where wireframe converges fast
    (64, 64, "wall", 100.0),
    (128, 128, "centre", 3.0),
    (256, 256, "wall", 1000.0),
    (128, 64, "wall", 30.0),
    (96, 136, "centre", 2.0),
    (512, 512, "wall", 300.0),
]


def _problem(mg, k, nx, ny, kind, ratio):
    import torch
    x = I.coords(nx, kind, ratio=ratio)
    y = I.coords(ny, "wall" if kind == "centre" else kind, ratio=ratio)
    f = torch.tensor(I.rhs_gaussian(ny + 1, nx + 1, 30 + k), device="cuda")
    g = np.random.default_rng(40 + k).standard_normal((ny + 1, nx + 1)) * (k % 2)  # some with boundary data
    g[1:-1, 1:-1] = 0.0
    return mg.Grid(x, y), f, torch.tensor(g, device="cuda")


def _kw(pr, precision):
    # the paper's pairing (Sec. 6): tweed for wall clustering, wireframe for
    # clustering towards the centre
    return dict(smoother="wireframe" if pr[2] == "centre" else "tweed", nu1=1, nu2=1, tol=1e-10,
                precision=precision, max_cycles=100, max_outer=25)


@pytest.mark.parametrize("precision", ["f64", "f32_refine"])
def test_batch_equals_individual_solves(mg, precision):
    import torch
    probs = [_problem(mg, k, *pr) for k, pr in enumerate(PROBLEMS)]
    grids = [p[0] for p in probs]
    params = [mg.default_params(**_kw(pr, precision)) for pr in PROBLEMS]
    us = [p[2].clone() for p in probs]
    res_b = mg.Batch(grids).solve(us, [p[1] for p in probs], params)
    torch.cuda.synchronize()
    for k, (grid, f, g) in enumerate(probs):
        u1 = g.clone()
        r1 = grid.solve(u1, f, **_kw(PROBLEMS[k], precision))
        info = (k, PROBLEMS[k], res_b[k], r1)
        assert res_b[k].status == r1.status == mg.OK, info
        assert res_b[k].cycles == r1.cycles and res_b[k].outer_iters == r1.outer_iters, info
        assert np.array_equal(res_b[k].history, r1.history), info
        assert torch.equal(us[k], u1), (info, float((us[k] - u1).abs().max()))


def test_batch_rejects_repeated_grid(mg):
    grid, _, _ = _problem(mg, 0, 16, 16, "wall", 10.0)
    with pytest.raises(mg.MGError):
        mg.Batch([grid, grid])
