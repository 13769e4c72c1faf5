"""Plain FP64 CPU oracle for tweed / wireframe multigrid (arXiv:2110.08389).

TEST INFRASTRUCTURE ONLY.  The product package never imports this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do.  The arithmetic lives in ``mg_oracle.c`` (plain C, FP64), which
shares no code with the CUDA path; this file only compiles it with gcc and
marshals arrays through ctypes.  The two-grid spectral radius (Sec. 5,
Eq. Mh2h) uses SciPy's ARPACK wrapper on the oracle's two-grid cycle as the
library eigen-solver step.

Every function pinned by the ``-m "not gpu"`` tests; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_SRC3 = os.path.join(_HERE, "mg_oracle3d.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmgoracle.so")
_lock = threading.Lock()
_lib = None

# Smoother and restriction codes (same numbering as the C file).
CHECKERBOARD, ZEBRA_X, ZEBRA_Y, ALT_ZEBRA, TWEED, WIREFRAME, ALT_TW = range(7)
HW, FW = 0, 1
POINT, PATH, CYCLE, STAR = range(4)
SMOOTHERS = {"checkerboard": CHECKERBOARD, "zebra_x": ZEBRA_X, "zebra_y": ZEBRA_Y,
             "alt_zebra": ALT_ZEBRA, "tweed": TWEED, "wireframe": WIREFRAME,
             "alt_tw": ALT_TW}


def build(force: bool = False) -> str:
    """Compile mg_oracle.c and mg_oracle3d.c into _build/libmgoracle.so (gcc,
    -O2, portable C11)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, _SRC3, "-lm"]
        # OpenMP over the decoupled blocks of a colour pass where the compiler
        # has it (same results with any thread count); plain C otherwise
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        i = ctypes.c_int
        d = ctypes.c_double
        sig = {
            "or_create": (P, [i, i, dp, dp]),
            "or_destroy": (None, [P]),
            "or_num_levels": (i, [P]),
            "or_threads": (i, [i]),
            "or_level_shape": (None, [P, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
            "or_level_coeffs": (None, [P, i, dp, dp, dp, dp]),
            "or_apply": (None, [P, i, dp, dp]),
            "or_residual": (None, [P, i, dp, dp, dp]),
            "or_colour_pass": (i, [P, i, i, i, dp, dp]),
            "or_smooth": (i, [P, i, i, dp, dp]),
            "or_restrict": (None, [P, i, i, dp, dp]),
            "or_prolong_add": (None, [P, i, dp, dp]),
            "or_direct_solve": (i, [P, i, dp, dp]),
            "or_cycle": (i, [P, i, i, i, i, i, dp, dp]),
            "or_solve": (i, [P, i, i, i, i, i, d, i, dp, dp, dp, dp, i]),
            "or_twogrid_apply": (i, [P, i, i, i, i, dp]),
            "or_partition_info": (i, [P, i, i, ip, i]),
            "or_partition_owner": (i, [P, i, i, ip]),
            "or_block_nodes": (i, [P, i, i, i, ip]),
            "or_block_dense": (i, [P, i, i, i, dp, dp, dp, dp]),
            "or_block_solve": (i, [P, i, i, i, dp, dp]),
            "or_dense_solve": (i, [i, dp, dp]),
            "o3_create": (P, [i, i, i, dp, dp, dp]),
            "o3_destroy": (None, [P]),
            "o3_num_levels": (i, [P]),
            "o3_level_shape": (None, [P, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
            "o3_level_coeffs": (None, [P, i, dp, dp, dp, dp, dp, dp]),
            "o3_apply": (None, [P, i, dp, dp]),
            "o3_residual": (None, [P, i, dp, dp, dp]),
            "o3_colour_pass": (i, [P, i, i, i, dp, dp]),
            "o3_smooth": (i, [P, i, i, dp, dp]),
            "o3_restrict": (None, [P, i, dp, dp]),
            "o3_prolong_add": (None, [P, i, dp, dp]),
            "o3_direct_solve": (i, [P, i, dp, dp]),
            "o3_partition": (i, [P, i, i, ip, ip, i]),
            "o3_block_solve": (i, [P, i, i, i, dp, dp]),
            "o3_cycle": (i, [P, i, i, i, dp, dp]),
            "o3_solve": (i, [P, i, i, i, d, i, dp, dp, dp, i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def threads(n: int = 0) -> int:
    """Threads of the oracle's colour passes (OpenMP builds; n <= 0 keeps the
    count).  Returns the count in effect (1 for a plain build)."""
    return int(_load().or_threads(int(n)))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Level hierarchy of Eq. (prob:DP) on the grid x (nx+1 nodes) by y (ny+1).

    Arrays are float64 of shape (ny+1, nx+1), x fastest; index 0 of the level
    list is the finest grid (the paper's Omega_p).
    """

    def __init__(self, x, y):
        self.lib = _load()
        self.x = _f64(x)
        self.y = _f64(y)
        self.nx = len(self.x) - 1
        self.ny = len(self.y) - 1
        self.h = self.lib.or_create(self.nx, self.ny, self.x, self.y)
        if not self.h:
            raise ValueError("oracle: bad grid")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    # ---- hierarchy
    @property
    def nlev(self) -> int:
        return self.lib.or_num_levels(self.h)

    def shape(self, lev: int = 0):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        self.lib.or_level_shape(self.h, lev, ctypes.byref(nx), ctypes.byref(ny))
        return ny.value + 1, nx.value + 1

    def coeffs(self, lev: int = 0):
        ny1, nx1 = self.shape(lev)
        W, E = np.zeros(nx1), np.zeros(nx1)
        S, N = np.zeros(ny1), np.zeros(ny1)
        self.lib.or_level_coeffs(self.h, lev, W, E, S, N)
        return W, E, S, N

    def zeros(self, lev: int = 0):
        return np.zeros(self.shape(lev))

    # ---- operator
    def apply(self, u, lev: int = 0):
        u = _f64(u)
        out = np.empty_like(u)
        self.lib.or_apply(self.h, lev, u, out)
        return out

    def residual(self, u, f, lev: int = 0):
        u, f = _f64(u), _f64(f)
        d = np.empty_like(u)
        self.lib.or_residual(self.h, lev, u, f, d)
        return d

    # ---- smoothing (in place on u)
    def colour_pass(self, u, f, smoother, colour, lev: int = 0):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        rc = self.lib.or_colour_pass(self.h, lev, SMOOTHERS.get(smoother, smoother), colour, u, _f64(f))
        if rc:
            raise RuntimeError("oracle colour pass failed")
        return u

    def smooth(self, u, f, smoother, steps: int = 1, lev: int = 0):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        f = _f64(f)
        for _ in range(steps):
            if self.lib.or_smooth(self.h, lev, SMOOTHERS.get(smoother, smoother), u, f):
                raise RuntimeError("oracle smoothing failed")
        return u

    # ---- transfers
    def restrict(self, d, kind=FW, lev: int = 0):
        fc = self.zeros(lev + 1)
        self.lib.or_restrict(self.h, lev, kind, _f64(d), fc)
        return fc

    def prolong_add(self, uc, u, lev: int = 0):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        self.lib.or_prolong_add(self.h, lev, _f64(uc), u)
        return u

    # ---- solves
    def direct_solve(self, u, f, lev: int = 0):
        """Dense-LU solution of the whole level (boundary values taken from u)."""
        u = _f64(u).copy()
        if self.lib.or_direct_solve(self.h, lev, u, _f64(f)):
            raise RuntimeError("singular system")
        return u

    def cycle(self, u, f, smoother="tweed", nu1=2, nu2=2, gamma=1, restriction=FW):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if self.lib.or_cycle(self.h, SMOOTHERS.get(smoother, smoother), nu1, nu2, gamma, restriction, u, _f64(f)):
            raise RuntimeError("oracle cycle failed")
        return u

    def solve(self, u, f, smoother="tweed", nu1=2, nu2=2, gamma=1, restriction=FW,
              tol=1e-10, max_cycles=100):
        """Cycles until ||f-Lu||_2/||f||_2 <= tol.  Returns (u, hist, hmax)."""
        u = _f64(u).copy()
        cap = max_cycles + 1
        hist, hmax = np.zeros(cap), np.zeros(cap)
        k = self.lib.or_solve(self.h, SMOOTHERS.get(smoother, smoother), nu1, nu2, gamma, restriction,
                              float(tol), int(max_cycles), u, _f64(f), hist, hmax, cap)
        if k < 0:
            raise RuntimeError("oracle solve failed")
        return u, hist[: k + 1].copy(), hmax[: k + 1].copy()

    # ---- two-grid analysis (Sec. 5)
    def twogrid_apply(self, e, smoother, restriction=FW, nu1=1, nu2=0):
        e = _f64(e).copy()
        if self.lib.or_twogrid_apply(self.h, SMOOTHERS.get(smoother, smoother), restriction, nu1, nu2, e):
            raise RuntimeError("two-grid apply failed")
        return e

    def twogrid_radius(self, smoother, restriction=FW, nu1=1, nu2=0, tol=1e-9, seed=0):
        """Spectral radius of Eq. (Mh2h) by ARPACK on the interior unknowns."""
        from scipy.sparse.linalg import LinearOperator, eigs

        ny1, nx1 = self.shape(0)
        n = (ny1 - 2) * (nx1 - 2)
        sm = SMOOTHERS.get(smoother, smoother)

        def mv(v):
            e = np.zeros((ny1, nx1))
            e[1:-1, 1:-1] = np.real(v).reshape(ny1 - 2, nx1 - 2)
            out = self.twogrid_apply(e, sm, restriction, nu1, nu2)
            return out[1:-1, 1:-1].ravel()

        if n <= 400:  # small grids: eigenvalues of the explicitly built matrix
            M = np.stack([mv(col) for col in np.eye(n)], axis=1)
            return float(np.max(np.abs(np.linalg.eigvals(M))))
        op = LinearOperator((n, n), matvec=mv, dtype=np.float64)
        v0 = np.random.default_rng(seed).standard_normal(n)
        # several eigenvalues at once: the dominant ones often come in close
        # pairs, which a single-eigenvalue Arnoldi run resolves poorly
        vals = eigs(op, k=6, which="LM", tol=tol, v0=v0, return_eigenvectors=False, ncv=40, maxiter=5000)
        return float(np.max(np.abs(vals)))

    # ---- partition inspection
    def partition(self, smoother, lev: int = 0):
        ny1, nx1 = self.shape(lev)
        cap = ny1 * nx1
        info = np.zeros(4 * cap, dtype=np.int32)
        nb = self.lib.or_partition_info(self.h, lev, SMOOTHERS.get(smoother, smoother), info, cap)
        if nb < 0:
            raise RuntimeError("partition failed")
        return info[: 4 * nb].reshape(nb, 4)  # (type, colour, size, legs)

    def owner(self, smoother, lev: int = 0):
        ny1, nx1 = self.shape(lev)
        o = np.zeros(ny1 * nx1, dtype=np.int32)
        if self.lib.or_partition_owner(self.h, lev, SMOOTHERS.get(smoother, smoother), o):
            raise RuntimeError("partition failed")
        return o.reshape(ny1, nx1)

    def block_nodes(self, smoother, b, lev: int = 0):
        ny1, nx1 = self.shape(lev)
        nodes = np.zeros(ny1 * nx1, dtype=np.int32)
        n = self.lib.or_block_nodes(self.h, lev, SMOOTHERS.get(smoother, smoother), b, nodes)
        nodes = nodes[:n]
        return [(int(p % nx1), int(p // nx1)) for p in nodes]  # (i, j)

    def block_dense(self, smoother, b, u, f, lev: int = 0):
        n = len(self.block_nodes(smoother, b, lev))
        A = np.zeros(n * n)
        r = np.zeros(n)
        self.lib.or_block_dense(self.h, lev, SMOOTHERS.get(smoother, smoother), b, _f64(u), _f64(f), A, r)
        return A.reshape(n, n), r

    def block_solve(self, smoother, b, u, f, lev: int = 0):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        self.lib.or_block_solve(self.h, lev, SMOOTHERS.get(smoother, smoother), b, u, _f64(f))
        return u


def dense_solve(A, b):
    """Gaussian elimination with partial pivoting (the oracle's own)."""
    A = _f64(A).copy().ravel()
    x = _f64(b).copy()
    if _load().or_dense_solve(len(x), A, x):
        raise RuntimeError("singular")
    return x


# ---- gradient through the solve (the adjoint; the paper has none)

def quadratic_loss_gradient(P: Problem, f, g, u_target):
    """Gradient of l(u) = 0.5 ||u - u_target||^2 (sum over all nodes), u the
    solution of Eq. (prob:DP) with source f inside and Dirichlet data g on the
    boundary, with respect to f (interior entries) and g (boundary entries).

    The plain definition, for small grids: with A the interior operator and B
    its coupling to the boundary values (both assembled by applying the
    oracle's operator to unit vectors), u_int = A^{-1} (f_int - B g_b),
    lambda = A^{-T} (u - u_target)_int, dl/df = lambda and
    dl/dg_b = (u - u_target)_b - (B^T lambda)_b.  Dense solves by the oracle's
    own Gaussian elimination.  Returns (l, u, grad_f, grad_g)."""
    ny1, nx1 = P.shape()
    f, g, ut = _f64(f), _f64(g), _f64(u_target)
    inner = np.zeros((ny1, nx1), dtype=bool)
    inner[1:-1, 1:-1] = True
    ii = np.flatnonzero(inner.ravel())
    bb = np.flatnonzero(~inner.ravel())
    n = len(ii)
    A = np.zeros((n, n))
    B = np.zeros((n, len(bb)))
    e = np.zeros(ny1 * nx1)
    for k, p in enumerate(ii):
        e[p] = 1.0
        A[:, k] = P.apply(e.reshape(ny1, nx1)).ravel()[ii]
        e[p] = 0.0
    for k, p in enumerate(bb):
        e[p] = 1.0
        B[:, k] = P.apply(e.reshape(ny1, nx1)).ravel()[ii]
        e[p] = 0.0
    gb = g.ravel()[bb]
    u = g.copy().ravel()
    u[ii] = dense_solve(A, f.ravel()[ii] - B @ gb)
    r = u - ut.ravel()
    lam = dense_solve(A.T.copy(), r[ii])
    grad_f = np.zeros(ny1 * nx1)
    grad_f[ii] = lam
    grad_g = np.zeros(ny1 * nx1)
    grad_g[bb] = r[bb] - B.T @ lam
    loss = 0.5 * float(r @ r)
    return loss, u.reshape(ny1, nx1), grad_f.reshape(ny1, nx1), grad_g.reshape(ny1, nx1)


SMOOTHERS3 = {"tweed": 0, "wireframe": 1, "complementary": 2, "alt_tw": 3, "triplet": 4}


class Problem3:
    """3D tweed / wireframe multigrid oracle (mg_oracle3d.c, Sec. 7) for the
    Dirichlet problem of Eq. (prob:DP) with a third axis.  Arrays are
    (nz+1, ny+1, nx+1), x fastest; only interior values of f and boundary
    values of u are read."""

    def __init__(self, x, y, z):
        self.lib = _load()
        self.x, self.y, self.z = _f64(x), _f64(y), _f64(z)
        self.h = self.lib.o3_create(len(self.x) - 1, len(self.y) - 1, len(self.z) - 1, self.x, self.y, self.z)
        if not self.h:
            raise ValueError("grid too small")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.o3_destroy(self.h)
            self.h = None

    @property
    def nlev(self) -> int:
        return self.lib.o3_num_levels(self.h)

    def dims(self, lev: int = 0):
        nx, ny, nz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.lib.o3_level_shape(self.h, lev, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz))
        return nx.value, ny.value, nz.value

    def shape(self, lev: int = 0):
        nx, ny, nz = self.dims(lev)
        return nz + 1, ny + 1, nx + 1

    def coeffs(self, lev: int = 0):
        nx, ny, nz = self.dims(lev)
        a = [np.zeros(nx + 1), np.zeros(nx + 1), np.zeros(ny + 1), np.zeros(ny + 1), np.zeros(nz + 1), np.zeros(nz + 1)]
        self.lib.o3_level_coeffs(self.h, lev, *a)
        return dict(zip("WESNBT", a))

    def apply(self, u, lev: int = 0):
        u = _f64(u)
        out = np.empty_like(u)
        self.lib.o3_apply(self.h, lev, u, out)
        return out

    def residual(self, u, f, lev: int = 0):
        u, f = _f64(u), _f64(f)
        d = np.empty_like(u)
        self.lib.o3_residual(self.h, lev, u, f, d)
        return d

    def colour_pass(self, u, f, colour, lev: int = 0, smoother="tweed"):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if self.lib.o3_colour_pass(self.h, lev, SMOOTHERS3[smoother], colour, u, _f64(f)):
            raise RuntimeError("oracle colour pass failed")
        return u

    def smooth(self, u, f, lev: int = 0, smoother="tweed"):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if self.lib.o3_smooth(self.h, lev, SMOOTHERS3[smoother], u, _f64(f)):
            raise RuntimeError("oracle smoothing failed")
        return u

    def restrict(self, d, lev: int = 0):
        fc = np.zeros(self.shape(lev + 1))
        self.lib.o3_restrict(self.h, lev, _f64(d), fc)
        return fc

    def prolong_add(self, uc, u, lev: int = 0):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        self.lib.o3_prolong_add(self.h, lev, _f64(uc), u)
        return u

    def direct_solve(self, u, f, lev: int = 0):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if self.lib.o3_direct_solve(self.h, lev, u, _f64(f)):
            raise RuntimeError("singular")
        return u

    def partition(self, lev: int = 0, smoother="tweed"):
        """(owner of every node, -1 off the interior; colour of every block)."""
        owner = np.empty(self.shape(lev), dtype=np.int32)
        cap = owner.size
        colour = np.empty(cap, dtype=np.int32)
        nb = self.lib.o3_partition(self.h, lev, SMOOTHERS3[smoother], owner, colour, cap)
        return owner, colour[:nb].copy()

    def block_solve(self, b, u, f, lev: int = 0, smoother="tweed"):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if self.lib.o3_block_solve(self.h, lev, SMOOTHERS3[smoother], b, u, _f64(f)):
            raise RuntimeError("block solve failed")
        return u

    def cycle(self, u, f, nu1=2, nu2=2, smoother="tweed"):
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if self.lib.o3_cycle(self.h, SMOOTHERS3[smoother], nu1, nu2, u, _f64(f)):
            raise RuntimeError("oracle cycle failed")
        return u

    def solve(self, u, f, nu1=2, nu2=2, tol=1e-10, max_cycles=100, cap=256, smoother="tweed"):
        """Cycles until tol; returns the relative-residual history."""
        assert u.dtype == np.float64 and u.flags.c_contiguous
        hist = np.zeros(cap)
        k = self.lib.o3_solve(self.h, SMOOTHERS3[smoother], nu1, nu2, tol, max_cycles, u, _f64(f), hist, cap)
        if k < 0:
            raise RuntimeError("oracle solve failed")
        return hist[:min(k, cap - 1) + 1].copy()
