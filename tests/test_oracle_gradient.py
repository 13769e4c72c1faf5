"""Pins of the oracle's gradient through the solve (the adjoint that the
autograd path is checked against): central differences of the quadratic loss
are exact up to rounding, so they fix the gradient independently of the
transpose solve used inside."""
import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I


def _loss(P, f, g, ut):
    u = P.direct_solve(g, f)
    r = u - ut
    return 0.5 * float(np.sum(r * r))


@pytest.mark.parametrize("nx,ny,kind", [(8, 6, "wall"), (10, 12, "centre")])
def test_gradient_matches_central_differences(oracle_mod, nx, ny, kind):
    x = I.coords(nx, kind, c=1.5)
    y = I.coords(ny, "wall", c=2.0)
    P = oracle_mod.Problem(x, y)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(P.shape())
    g = I.random_field(*P.shape(), seed=4)
    g = rng.standard_normal(P.shape()) - g  # nonzero boundary data
    ut = rng.standard_normal(P.shape())
    loss, u, gf, gg = oracle_mod.quadratic_loss_gradient(P, f, g, ut)
    assert loss == pytest.approx(_loss(P, f, g, ut), rel=1e-12)
    inner = np.zeros(P.shape(), dtype=bool)
    inner[1:-1, 1:-1] = True
    for s in range(6):
        d = rng.standard_normal(P.shape())
        h = 1.0  # the loss is quadratic in f and g: central differences are exact
        df = np.where(inner, d, 0.0)
        fd = (_loss(P, f + h * df, g, ut) - _loss(P, f - h * df, g, ut)) / (2 * h)
        assert fd == pytest.approx(np.sum(gf * df), rel=1e-7, abs=1e-9 * abs(loss))
        dg = np.where(inner, 0.0, d)
        fd = (_loss(P, f, g + h * dg, ut) - _loss(P, f, g - h * dg, ut)) / (2 * h)
        assert fd == pytest.approx(np.sum(gg * dg), rel=1e-7, abs=1e-9 * abs(loss))
    # entries that do not enter the problem get no gradient
    assert np.all(gf[~inner] == 0.0) and np.all(gg[inner] == 0.0)
