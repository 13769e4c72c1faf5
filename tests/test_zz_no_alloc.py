"""mg_residual_norm_static: the norm entry point for callers that cannot
allocate device memory (its scratch is a static device array).  Checked
against the norm the solver itself reports, on two calls in a row.  This file
is collected last so that a failure here cannot hide any other test."""
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


def test_static_norm_rejects_oversize(mg):
    import torch
    lib = mg.load()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    st = lib.mg_residual_norm_static(8, 16386, p, p, p, p, p, p, p, None)
    assert st == mg.ERR_SIZE
    assert b"static scratch" in lib.mg_last_error()
