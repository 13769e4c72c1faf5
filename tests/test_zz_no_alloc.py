"""mg_residual_norm_static: the norm entry point for callers that cannot
allocate device memory (its scratch is a static device array).  Checked
against the norm the solver itself reports and against a NumPy evaluation of
f - L u (nonzero boundary values included), on calls in a row.  This file is
collected last so that a failure here cannot hide any other test."""
import ctypes

import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def axis_coefficients(x):
    """Sec. 2: W_i = 1/(dx_i dx_{i-1/2}), E_i = 1/(dx_i dx_{i+1/2})."""
    lo, hi = np.zeros_like(x), np.zeros_like(x)
    dm = x[1:-1] - x[:-2]
    dp = x[2:] - x[1:-1]
    dc = 0.5 * (x[2:] - x[:-2])
    lo[1:-1] = 1.0 / (dc * dm)
    hi[1:-1] = 1.0 / (dc * dp)
    return lo, hi


def test_static_norm_matches_solver_norm(mg):
    import torch
    lib = mg.load()
    x = I.wall_coords(384, 3.0)
    y = I.centre_coords(256, 1.5)
    nx, ny = len(x) - 1, len(y) - 1
    W, E = axis_coefficients(x)
    S, N = axis_coefficients(y)
    dev = [torch.tensor(a, device="cuda") for a in (W, E, S, N)]
    grid = mg.Grid(x, y)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        # zero boundary data, so that the solver's scale ||f - B g|| is ||f||
        u_h = I.random_field(ny + 1, nx + 1, seed=100 + call)
        f_h = I.rhs_gaussian(ny + 1, nx + 1, seed=200 + call)
        u = torch.tensor(u_h, device="cuda")
        f = torch.tensor(f_h, device="cuda")
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.mg_residual_norm_static(nx, ny, *[ctypes.c_void_p(t.data_ptr()) for t in dev],
                                         ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == mg.OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        rel_static = np.sqrt(o[0] / o[2])
        # the existing path: mg_solve with the given u as initial guess and no
        # cycles reports the same relative defect from its own reduction
        res = grid.solve(u.clone(), f, smoother="tweed", use_initial_guess=1, max_cycles=0, tol=0.0)
        assert res.status == mg.ERR_NOT_CONVERGED and res.cycles == 0
        assert rel_static == pytest.approx(res.rel_res, rel=1e-12)
        assert o[2] == pytest.approx(np.sum(f_h[1:-1, 1:-1] ** 2), rel=1e-12)
        assert o[3] == np.abs(f_h[1:-1, 1:-1]).max()


def _call(lib, nx, ny, dev, u, f, out, stream):
    return lib.mg_residual_norm_static(nx, ny, *[ctypes.c_void_p(t.data_ptr()) for t in dev],
                                       ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def _numpy_defect(W, E, S, N, u, f):
    """f - L u of Eq. (prob:DP) at the interior nodes, written out in NumPy:
    every neighbour term, the boundary values of u included."""
    c = -(W[None, 1:-1] + E[None, 1:-1] + S[1:-1, None] + N[1:-1, None])
    lu = (W[None, 1:-1] * u[1:-1, :-2] + E[None, 1:-1] * u[1:-1, 2:]
          + S[1:-1, None] * u[:-2, 1:-1] + N[1:-1, None] * u[2:, 1:-1] + c * u[1:-1, 1:-1])
    return f[1:-1, 1:-1] - lu


def test_static_norm_with_boundary_data_matches_numpy(mg):
    """Nonzero boundary values, so the rows next to each wall read their
    boundary neighbours (i = 1, nx-1; j = 1, ny-1): all four outputs against
    NumPy and the defect of the existing mg_residual entry, on two calls."""
    import torch
    lib = mg.load()
    x = I.wall_coords(320, 2.0)
    y = I.centre_coords(200, 1.5)
    nx, ny = len(x) - 1, len(y) - 1
    W, E = axis_coefficients(x)
    S, N = axis_coefficients(y)
    dev = [torch.tensor(a, device="cuda") for a in (W, E, S, N)]
    grid = mg.Grid(x, y)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        rng = np.random.default_rng(300 + call)
        u_h = rng.standard_normal((ny + 1, nx + 1))  # boundary values included
        f_h = I.rhs_gaussian(ny + 1, nx + 1, seed=400 + call)
        u, f = torch.tensor(u_h, device="cuda"), torch.tensor(f_h, device="cuda")
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, nx, ny, dev, u, f, out, stream) == mg.OK
        d = torch.zeros_like(u)
        grid.residual(u, f, d)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        r = _numpy_defect(W, E, S, N, u_h, f_h)
        assert o[0] == pytest.approx(np.sum(r ** 2), rel=1e-12)
        assert o[1] == pytest.approx(np.abs(r).max(), rel=1e-12)
        assert o[2] == pytest.approx(np.sum(f_h[1:-1, 1:-1] ** 2), rel=1e-12)
        assert o[3] == np.abs(f_h[1:-1, 1:-1]).max()
        dd = d.cpu().numpy()[1:-1, 1:-1]
        assert o[0] == pytest.approx(np.sum(dd ** 2), rel=1e-12)
        assert o[1] == pytest.approx(np.abs(dd).max(), rel=1e-12)
    # a NaN in u reaches both residual norms, the maximum as well as the sum
    u_h[7, 9] = np.nan
    u = torch.tensor(u_h, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert _call(lib, nx, ny, dev, u, f, out, stream) == mg.OK
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.isnan(o[0]) and np.isnan(o[1]) and np.isfinite(o[2]) and np.isfinite(o[3])


def test_static_norm_rejects_oversize(mg):
    import torch
    lib = mg.load()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    st = lib.mg_residual_norm_static(8, 16386, p, p, p, p, p, p, p, None)
    assert st == mg.ERR_SIZE
    assert b"static scratch" in lib.mg_last_error()
