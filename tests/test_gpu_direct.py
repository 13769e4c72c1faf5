"""mg_direct_solve / mg_params.coarse_direct: the FP32 direct solve of one
coarse level (fast diagonalisation of the Kronecker-sum operator) against the
oracle's dense LU of that level, and FP32+refine solves that use it in their
cycles: same tolerance reached, solution equal to the FP64 solve's."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _xy(nx, ny, kind, ratio):
    return I.coords(nx, kind, ratio=ratio), I.coords(ny, "wall" if kind == "centre" else kind, ratio=ratio)


@pytest.mark.parametrize("nx,ny,kind,ratio", [(96, 64, "wall", 300.0), (128, 96, "wall", 1000.0),
                                              (256, 128, "centre", 10.0), (64, 256, "uniform", 1.0)])
def test_direct_solve_equals_dense_lu(mg, oracle_mod, nx, ny, kind, ratio):
    import torch
    x, y = (I.uniform_coords(nx), I.uniform_coords(ny)) if kind == "uniform" else _xy(nx, ny, kind, ratio)
    g = mg.Grid(x, y)
    P = oracle_mod.Problem(x, y)
    lev = g.direct_level
    assert lev >= 1 and max(g.shape(lev)) - 1 <= 64 and lev < g.nlev - 1
    if lev > 1:
        assert max(g.shape(lev - 1)) - 1 > 64
    rng = np.random.default_rng(21)
    shape = P.shape(lev)
    assert tuple(g.shape(lev)) == tuple(shape)
    f = rng.standard_normal(shape)
    u = rng.standard_normal(shape)  # boundary values enter the right-hand side
    u[1:-1, 1:-1] = 0.0
    u32 = u.astype(np.float32).astype(np.float64)
    f32 = f.astype(np.float32).astype(np.float64)
    ref = P.direct_solve(u32.copy(), f32, lev)
    ud = torch.tensor(u32, dtype=torch.float32, device="cuda")
    g.direct_solve(ud, torch.tensor(f32, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    got = ud.double().cpu().numpy()
    inner = (slice(1, -1), slice(1, -1))
    err = np.abs(got[inner] - ref[inner]).max() / np.abs(ref[inner]).max()
    assert err <= 2e-5, err
    assert np.array_equal(got[0], u32[0]) and np.array_equal(got[:, 0], u32[:, 0])


@pytest.mark.parametrize("smoother,kind,ratio", [("tweed", "wall", 1000.0), ("wireframe", "centre", 3.0)])
def test_refine_with_direct_level(mg, smoother, kind, ratio):
    import torch
    x, y = _xy(512, 512, kind, ratio)
    g = mg.Grid(x, y)
    f = torch.tensor(I.rhs_gaussian(513, 513, 22), device="cuda")
    kw = dict(smoother=smoother, nu1=1, nu2=1, tol=1e-10, max_outer=30, max_cycles=300)
    u64 = torch.zeros_like(f)
    r64 = g.solve(u64, f, precision="f64", **kw)
    u0 = torch.zeros_like(f)
    r0 = g.solve(u0, f, precision="f32_refine", **kw)
    u1 = torch.zeros_like(f)
    r1 = g.solve(u1, f, precision="f32_refine", coarse_direct=1, **kw)
    assert r64.status == r0.status == r1.status == mg.OK
    assert r1.rel_res <= 1e-10
    assert r1.outer_iters <= r0.outer_iters + 1
    err = float((u1 - u64).abs().max() / u64.abs().max())
    assert err <= 1e-9, err


def test_direct_level_batch_and_3d(mg):
    import torch
    grids = [mg.Grid(*_xy(256, 256, "wall", 300.0)), mg.Grid(*_xy(128, 128, "wall", 100.0))]
    fs = [torch.tensor(I.rhs_gaussian(257, 257, 23), device="cuda"), torch.tensor(I.rhs_gaussian(129, 129, 24), device="cuda")]
    kw = dict(smoother="tweed", nu1=1, nu2=1, tol=1e-10, precision="f32_refine", max_outer=20, max_cycles=200,
              coarse_direct=1)
    us = [torch.zeros_like(f) for f in fs]
    res = mg.Batch(grids).solve(us, fs, [mg.default_params(**kw) for _ in grids])
    torch.cuda.synchronize()
    for k in range(2):
        u1 = torch.zeros_like(fs[k])
        r1 = grids[k].solve(u1, fs[k], **kw)
        assert res[k].status == r1.status == mg.OK
        assert np.array_equal(res[k].history, r1.history)
        assert torch.equal(us[k], u1)
    z = I.coords(16, "wall", ratio=10.0)
    g3 = mg.Grid(z, z, z)
    assert g3.direct_level == -1
    u = torch.zeros(g3.shape(), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError) as e:
        g3.solve(u, u.clone() + 1, precision="f32_refine", coarse_direct=1)
    assert e.value.status == mg.ERR_UNSUPPORTED
