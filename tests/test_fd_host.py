"""Host part of the direct level solve (csrc/fd_host.h), on the CPU: the
symmetrised 1D factor of the operator and its Jacobi eigen-decomposition.
Pinned by orthogonality, by reconstructing the tridiagonal operator, by the
closed-form eigenvalues of the uniform grid (-4/h^2 sin^2(k pi / 2n)), and by
the fast-diagonalisation solve of a 2D level against a dense solve."""
import os
import subprocess

import numpy as np
import pytest

from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = tmp_path_factory.mktemp("fd") / "fd_host_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fd_host_driver.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def coefficients(x):
    """W_i, E_i of Sec. 2 on the interior nodes 1..n-1."""
    n = len(x) - 1
    dx = 0.5 * (x[2:] - x[:-2])
    W = 1.0 / (dx * (x[1:-1] - x[:-2]))
    E = 1.0 / (dx * (x[2:] - x[1:-1]))
    return n, W, E


def transforms(driver, x):
    n, W, E = coefficients(x)
    inp = f"{n}\n" + "\n".join(f"{v:.17g}" for v in W) + "\n" + "\n".join(f"{v:.17g}" for v in E) + "\n"
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout.split()
    m = n - 1
    vals = np.array([float(v) for v in out[1:]])
    assert out[0] == "1" and len(vals) == 2 * m + m * m
    return W, E, vals[:m], vals[m:2 * m], vals[2 * m:].reshape(m, m)


def tridiag(W, E):
    A = np.diag(-(W + E)) + np.diag(W[1:], -1) + np.diag(E[:-1], 1)
    return A


@pytest.mark.parametrize("kind,n,ratio", [("wall", 64, 1000.0), ("centre", 48, 50.0), ("wall", 16, 10.0)])
def test_eigen_decomposition_reconstructs_the_operator(driver, kind, n, ratio):
    x = I.coords(n, kind, ratio=ratio)
    W, E, lam, sd, Q = transforms(driver, x)
    assert np.abs(Q.T @ Q - np.eye(len(lam))).max() <= 1e-12
    A = tridiag(W, E)
    rec = (Q * lam) @ Q.T
    rec = rec / sd[:, None] * sd[None, :]
    assert np.abs(rec - A).max() <= 1e-12 * np.abs(A).max()
    assert (lam < 0).all()


def test_uniform_grid_eigenvalues_closed_form(driver):
    n = 32
    x = I.uniform_coords(n)
    _, _, lam, _, _ = transforms(driver, x)
    h = 1.0 / n
    k = np.arange(1, n)
    ref = -4.0 / h ** 2 * np.sin(k * np.pi / (2 * n)) ** 2
    assert np.allclose(np.sort(lam), np.sort(ref), rtol=1e-12, atol=0)


def test_fast_diagonalisation_solves_a_level(driver):
    """U = Dy^-1/2 Qy [(Qy^T Dy^1/2 R Dx^1/2 Qx) / (lx_i + ly_j)] Qx^T Dx^-1/2
    equals the dense solve of the Kronecker-sum operator."""
    x = I.coords(40, "wall", ratio=300.0)
    y = I.coords(24, "centre", ratio=20.0)
    Wx, Ex, lx, sx, Qx = transforms(driver, x)
    Wy, Ey, ly, sy, Qy = transforms(driver, y)
    Ax, Ay = tridiag(Wx, Ex), tridiag(Wy, Ey)
    my, mx = len(ly), len(lx)
    R = np.random.default_rng(1).standard_normal((my, mx))
    Rh = Qy.T @ (sy[:, None] * R * sx[None, :]) @ Qx
    U = Qy @ (Rh / (lx[None, :] + ly[:, None])) @ Qx.T / (sy[:, None] * sx[None, :])
    L = np.kron(np.eye(my), Ax) + np.kron(Ay, np.eye(mx))  # rows j*mx + i
    ref = np.linalg.solve(L, R.ravel()).reshape(my, mx)
    assert np.abs(U - ref).max() <= 1e-9 * np.abs(ref).max()
