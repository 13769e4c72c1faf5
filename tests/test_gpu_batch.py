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


PACKED = [  # (nx, ny, kind, ratio, nu1): equal shapes and parameters form packed groups
    (128, 128, "wall", 10.0, 1),
    (128, 128, "wall", 1000.0, 1),   # more refinement steps than its group partners
    (96, 136, "centre", 2.0, 1),
    (128, 128, "wall", 100.0, 1),    # zero data: converged at the initial residual, masked afterwards
    (96, 136, "centre", 1.5, 1),
    (128, 128, "wall", 100.0, 2),    # other parameters: solved on its own
    (256, 256, "wall", 300.0, 1),    # no partner of its shape: solved on its own
]


def test_packed_groups_equal_individual_solves(mg):
    """Problems of one shape and one parameter set run as packed groups (one
    launch per kernel for the whole group, members masked once converged);
    each result must still equal, bit for bit, mg_solve on the problem alone,
    and the batch must launch fewer kernels than the solves one by one."""
    import torch
    lib = mg.load()
    probs = [_problem(mg, k, nx, ny, kind, ratio) for k, (nx, ny, kind, ratio, _) in enumerate(PACKED)]
    probs[3] = (probs[3][0], torch.zeros_like(probs[3][1]), torch.zeros_like(probs[3][2]))
    grids = [p[0] for p in probs]

    def kw(k):
        nx, ny, kind, ratio, nu1 = PACKED[k]
        d = _kw((nx, ny, kind), "f32_refine")
        d["nu1"] = nu1
        return d

    params = [mg.default_params(**kw(k)) for k in range(len(PACKED))]
    us = [p[2].clone() for p in probs]
    batch = mg.Batch(grids)
    batch.solve(us, [p[1] for p in probs], params)  # first call captures the group graphs
    us = [p[2].clone() for p in probs]
    torch.cuda.synchronize()
    l0 = lib.mg_kernel_launches()
    res_b = batch.solve(us, [p[1] for p in probs], params)
    torch.cuda.synchronize()
    launches_batch = lib.mg_kernel_launches() - l0
    launches_single = 0
    for k, (grid, f, g) in enumerate(probs):
        u1 = g.clone()
        grid.solve(u1, f, **kw(k))  # graphs captured
        u1 = g.clone()
        torch.cuda.synchronize()
        l0 = lib.mg_kernel_launches()
        r1 = grid.solve(u1, f, **kw(k))
        torch.cuda.synchronize()
        launches_single += lib.mg_kernel_launches() - l0
        info = (k, PACKED[k], res_b[k], r1)
        assert res_b[k].status == r1.status == mg.OK, info
        assert res_b[k].cycles == r1.cycles and res_b[k].outer_iters == r1.outer_iters, info
        assert np.array_equal(res_b[k].history, r1.history), info
        assert torch.equal(us[k], u1), (info, float((us[k] - u1).abs().max()))
    outer = [r.outer_iters for r in res_b]
    assert outer[3] == 0 and min(outer[0], outer[1]) > 0  # members of one group stopped at different steps
    assert launches_batch < 0.75 * launches_single, (launches_batch, launches_single)


def test_unpackable_problem_in_batch(mg):
    """A grid whose line path is forced off the warp path on one level is
    solved on its own inside the batch, with the same result as alone."""
    import torch
    probs = [_problem(mg, k, 128, 128, "wall", 100.0) for k in range(3)]
    probs[1][0].set_line_path(1, "tweed", "f32", "cta")
    grids = [p[0] for p in probs]
    kw = _kw((128, 128, "wall"), "f32_refine")
    us = [p[2].clone() for p in probs]
    res_b = mg.Batch(grids).solve(us, [p[1] for p in probs], mg.default_params(**kw))
    for k, (grid, f, g) in enumerate(probs):
        u1 = g.clone()
        r1 = grid.solve(u1, f, **kw)
        assert res_b[k].status == r1.status == mg.OK
        assert np.array_equal(res_b[k].history, r1.history)
        assert torch.equal(us[k], u1)
