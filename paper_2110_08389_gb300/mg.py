"""Python binding of the tweedmg C ABI (``include/mg.h``).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libtweedmg.so``.  Arrays are torch CUDA tensors (float64 or float32,
contiguous, shape ``(ny+1, nx+1)``); streams default to torch's current
stream.  There is no CPU fallback: loading fails loudly when the library has
not been built (``python -m paper_2110_08389_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library to load: the checked build when TWEEDMG_LIB says so (build.py)
LIB_PATH = os.environ.get("TWEEDMG_LIB") or os.path.join(_HERE, "_build", "libtweedmg.so")

# enums (include/mg.h)
OK, ERR_INVALID_ARG, ERR_SIZE, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_TIMEOUT, ERR_ALLOC, \
    ERR_UNSUPPORTED = range(9)
CHECKERBOARD, ZEBRA_X, ZEBRA_Y, ALT_ZEBRA, TWEED, WIREFRAME, ALT_TW = range(7)
SMOOTHERS = {"checkerboard": CHECKERBOARD, "zebra_x": ZEBRA_X, "zebra_y": ZEBRA_Y, "alt_zebra": ALT_ZEBRA,
             "tweed": TWEED, "wireframe": WIREFRAME, "alt_tw": ALT_TW}
F64, F32 = 0, 1
PREC_F64, PREC_F32_REFINE = 0, 1
HW, FW = 0, 1
PATH_AUTO, PATH_WARP, PATH_TILED, PATH_CTA, PATH_CLUSTER = range(5)
PATHS = {"auto": PATH_AUTO, "warp": PATH_WARP, "tiled": PATH_TILED, "cta": PATH_CTA, "cluster": PATH_CLUSTER}
PATH_NAMES = {v: k for k, v in PATHS.items()}
DTYPES = {"f64": F64, "f32": F32}

# every symbol include/mg.h declares
EXPORTS = ["mg_setup_grid", "mg_destroy", "mg_num_levels", "mg_level_shape", "mg_smooth_tweed",
           "mg_smooth_wireframe", "mg_smooth", "mg_colour_pass", "mg_residual_restrict", "mg_prolong_add",
           "mg_residual", "mg_coarse_solve", "mg_vcycle", "mg_solve", "mg_solve_adjoint",
           "mg_default_params", "mg_status_string", "mg_last_error", "mg_kernel_launches",
           "mg_residual_norm_static", "mg_pass_timer_begin", "mg_pass_timer_end", "mg_boundary_adjoint", "mg_batch_create",
           "mg_batch_destroy", "mg_batch_solve", "mg_set_line_path", "mg_get_line_path", "mg_autotune",
           "mg_level_dims", "mg_grid_dim", "mg_direct_level", "mg_direct_solve", "mg_check_word"]


class MGError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: status {status} ({detail})")


class Params(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("cycle", ctypes.c_int), ("restriction", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("max_outer", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("use_initial_guess", ctypes.c_int), ("early_stop", ctypes.c_int), ("coarse_direct", ctypes.c_int),
                ("tol", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer_iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("conv_factor", ctypes.c_double), ("ms", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int),
                ("history_len", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing -- no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"tweedmg CUDA library not built: {path} missing "
                           "(run python -m paper_2110_08389_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, i, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "mg_setup_grid": (i, [ctypes.POINTER(vp), i, i64p, ctypes.POINTER(ctypes.c_void_p), i, vp]),
        "mg_destroy": (None, [vp]),
        "mg_num_levels": (i, [vp]),
        "mg_level_shape": (i, [vp, i, i64p, i64p]),
        "mg_smooth_tweed": (i, [vp, i, vp, vp, i, i, vp]),
        "mg_smooth_wireframe": (i, [vp, i, vp, vp, i, i, vp]),
        "mg_smooth": (i, [vp, i, i, vp, vp, i, i, vp]),
        "mg_colour_pass": (i, [vp, i, i, i, vp, vp, i, vp]),
        "mg_residual_restrict": (i, [vp, i, i, vp, vp, vp, vp, i, vp]),
        "mg_prolong_add": (i, [vp, i, vp, vp, i, vp]),
        "mg_residual": (i, [vp, i, vp, vp, vp, i, vp]),
        "mg_coarse_solve": (i, [vp, vp, vp, i, vp]),
        "mg_direct_level": (i, [vp]),
        "mg_direct_solve": (i, [vp, vp, vp, vp]),
        "mg_vcycle": (i, [vp, vp, vp, ctypes.POINTER(Params), vp]),
        "mg_solve": (i, [vp, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(Info), vp]),
        "mg_solve_adjoint": (i, [vp, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(Info), vp]),
        "mg_default_params": (None, [ctypes.POINTER(Params)]),
        "mg_status_string": (ctypes.c_char_p, [i]),
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_kernel_launches": (ctypes.c_ulonglong, []),
        "mg_residual_norm_static": (i, [ctypes.c_int64, ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]),
        "mg_pass_timer_begin": (i, [vp, i, i]),
        "mg_boundary_adjoint": (i, [vp, vp, vp, vp, vp]),
        "mg_batch_create": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]),
        "mg_batch_destroy": (None, [vp]),
        "mg_batch_solve": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(Params), i,
                               ctypes.POINTER(Info), ctypes.POINTER(ctypes.c_int), vp]),
        "mg_pass_timer_end": (i, [vp, i64p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
        "mg_set_line_path": (i, [vp, i, i, i, i, i]),
        "mg_get_line_path": (i, [vp, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "mg_autotune": (i, [vp, i, i, i, ctypes.POINTER(ctypes.c_double), vp]),
        "mg_level_dims": (i, [vp, i, i64p]),
        "mg_grid_dim": (i, [vp]),
        "mg_check_word": (ctypes.c_uint, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, what: str, ok=(OK,)):
    if st not in ok:
        lib = load()
        raise MGError(st, what, f"{lib.mg_status_string(st).decode()}; {lib.mg_last_error().decode()}")
    return st


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError("tweedmg arrays are float64 or float32")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tweedmg arrays must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class SolveResult:
    status: int
    cycles: int
    outer_iters: int
    rel_res: float
    conv_factor: float
    ms: float
    history: np.ndarray


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().mg_kernel_launches())


def default_params(**kw) -> Params:
    """mg_default_params() with fields overridden by keyword: smoother (name or
    code), nu1, nu2, cycle ("V"/"W"), restriction ("hw"/"fw"), precision
    ("f64"/"f32_refine"), max_cycles, max_outer, inner_cycles,
    use_initial_guess, early_stop (give up once the last step's rate cannot
    reach tol within the caps), coarse_direct (FP32 cycles solve the direct
    level exactly), tol."""
    p = Params()
    load().mg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "smoother" and isinstance(v, str):
            v = SMOOTHERS[v]
        if k == "precision" and isinstance(v, str):
            v = {"f64": PREC_F64, "f32_refine": PREC_F32_REFINE}[v]
        if k == "restriction" and isinstance(v, str):
            v = {"hw": HW, "fw": FW}[v.lower()]
        if k == "cycle" and isinstance(v, str):
            v = {"V": 1, "W": 2}[v.upper()]
        setattr(p, k, v)
    return p


class Grid:
    """mg_setup_grid on host coordinate arrays x (nx+1) and y (ny+1), and z
    (nz+1) for a 3D grid (Sec. 7; arrays then have shape (nz+1, ny+1, nx+1))."""

    def __init__(self, x, y, z=None, precision_mask: int = 3, stream=None):
        self.lib = load()
        axes = [np.ascontiguousarray(a, dtype=np.float64) for a in ((x, y) if z is None else (x, y, z))]
        self.x, self.y = axes[0], axes[1]
        self.z = axes[2] if z is not None else None
        self.dim = len(axes)
        n = (ctypes.c_int64 * self.dim)(*[len(a) - 1 for a in axes])
        coords = (ctypes.c_void_p * self.dim)(*[a.ctypes.data for a in axes])
        h = ctypes.c_void_p()
        _check(self.lib.mg_setup_grid(ctypes.byref(h), self.dim, n, coords, precision_mask,
                                      _stream(stream) if stream is not None else None), "mg_setup_grid")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nlev(self) -> int:
        return self.lib.mg_num_levels(self.h)

    def shape(self, level: int = 0):
        """Array shape of a level: (ny+1, nx+1), or (nz+1, ny+1, nx+1) in 3D."""
        d = (ctypes.c_int64 * 3)()
        _check(self.lib.mg_level_dims(self.h, level, d), "mg_level_dims")
        if self.dim == 3:
            return d[2] + 1, d[1] + 1, d[0] + 1
        return d[1] + 1, d[0] + 1

    # ---- relaxation
    def smooth(self, u, f, smoother="tweed", sweeps=1, level=0, stream=None):
        sm = SMOOTHERS[smoother] if isinstance(smoother, str) else smoother
        _check(self.lib.mg_smooth(self.h, level, sm, _ptr(u), _ptr(f), sweeps, _dtype_code(u), _stream(stream)),
               "mg_smooth")
        return u

    def smooth_tweed(self, u, f, sweeps=1, level=0, stream=None):
        _check(self.lib.mg_smooth_tweed(self.h, level, _ptr(u), _ptr(f), sweeps, _dtype_code(u), _stream(stream)),
               "mg_smooth_tweed")
        return u

    def smooth_wireframe(self, u, f, sweeps=1, level=0, stream=None):
        _check(self.lib.mg_smooth_wireframe(self.h, level, _ptr(u), _ptr(f), sweeps, _dtype_code(u),
                                            _stream(stream)), "mg_smooth_wireframe")
        return u

    def colour_pass(self, u, f, smoother="tweed", colour=0, level=0, stream=None):
        sm = SMOOTHERS[smoother] if isinstance(smoother, str) else smoother
        _check(self.lib.mg_colour_pass(self.h, level, sm, colour, _ptr(u), _ptr(f), _dtype_code(u),
                                       _stream(stream)), "mg_colour_pass")
        return u

    # ---- line-solve paths (mg_set_line_path / mg_get_line_path / mg_autotune)
    def set_line_path(self, level, smoother="tweed", dtype="f32", path="warp", k=0):
        """Force the line-solve path of one level; raises MGError with status
        ERR_UNSUPPORTED when the level's blocks do not fit it."""
        sm = SMOOTHERS[smoother] if isinstance(smoother, str) else smoother
        dt = DTYPES[dtype] if isinstance(dtype, str) else dtype
        pa = PATHS[path] if isinstance(path, str) else path
        _check(self.lib.mg_set_line_path(self.h, level, sm, dt, pa, k), "mg_set_line_path")

    def line_path(self, level, smoother="tweed", dtype="f32"):
        """(path name, nodes per thread, warps per sequence) of one level."""
        sm = SMOOTHERS[smoother] if isinstance(smoother, str) else smoother
        dt = DTYPES[dtype] if isinstance(dtype, str) else dtype
        p, k, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.mg_get_line_path(self.h, level, sm, dt, ctypes.byref(p), ctypes.byref(k), ctypes.byref(w)),
               "mg_get_line_path")
        return PATH_NAMES[p.value], k.value, w.value

    def autotune(self, smoother="tweed", dtype="f32", reps=20, stream=None):
        """Time every path and warp shape per level, keep the fastest; returns
        the chosen microseconds per colour pass per level."""
        sm = SMOOTHERS[smoother] if isinstance(smoother, str) else smoother
        dt = DTYPES[dtype] if isinstance(dtype, str) else dtype
        t = (ctypes.c_double * self.nlev)()
        _check(self.lib.mg_autotune(self.h, sm, dt, reps, t, _stream(stream)), "mg_autotune")
        return [float(v) for v in t]

    def boundary_adjoint(self, lam, grad_u, grad_g, stream=None):
        """grad_g from the adjoint state lam and dloss/du (mg_boundary_adjoint)."""
        _check(self.lib.mg_boundary_adjoint(self.h, _ptr(lam), _ptr(grad_u), _ptr(grad_g), _stream(stream)),
               "mg_boundary_adjoint")
        return grad_g

    def pass_timer_begin(self, level=0, max_passes=4096):
        """Time every colour pass on `level` from now on with CUDA events on
        its stream (mg_pass_timer_begin)."""
        _check(self.lib.mg_pass_timer_begin(self.h, level, max_passes), "mg_pass_timer_begin")

    def pass_timer_end(self) -> dict:
        """Stop the timer: passes timed, summed ms per stage (reduce, couple,
        expand) and the fastest / slowest pass (mg_pass_timer_end)."""
        n = ctypes.c_int64()
        st = (ctypes.c_double * 3)()
        mn, mx = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.mg_pass_timer_end(self.h, ctypes.byref(n), st, ctypes.byref(mn), ctypes.byref(mx)),
               "mg_pass_timer_end")
        return {"passes": int(n.value), "stage_ms": [float(v) for v in st], "pass_min_ms": float(mn.value),
                "pass_max_ms": float(mx.value)}

    # ---- transfers
    def residual(self, u, f, d, level=0, stream=None):
        _check(self.lib.mg_residual(self.h, level, _ptr(u), _ptr(f), _ptr(d), _dtype_code(u), _stream(stream)),
               "mg_residual")
        return d

    def residual_restrict(self, u, f, fc, uc=None, restriction=FW, level=0, stream=None):
        _check(self.lib.mg_residual_restrict(self.h, level, restriction, _ptr(u), _ptr(f), _ptr(fc), _ptr(uc),
                                             _dtype_code(u), _stream(stream)), "mg_residual_restrict")
        return fc

    def prolong_add(self, uc, u, level=0, stream=None):
        _check(self.lib.mg_prolong_add(self.h, level, _ptr(uc), _ptr(u), _dtype_code(u), _stream(stream)),
               "mg_prolong_add")
        return u

    def coarse_solve(self, u, f, stream=None):
        _check(self.lib.mg_coarse_solve(self.h, _ptr(u), _ptr(f), _dtype_code(u), _stream(stream)),
               "mg_coarse_solve")
        return u

    @property
    def direct_level(self) -> int:
        """Level the FP32 cycles solve directly under coarse_direct=1 (-1: none)."""
        return int(self.lib.mg_direct_level(self.h))

    def direct_solve(self, u, f, stream=None):
        """FP32 direct solve of the direct level's interior system (in place)."""
        _check(self.lib.mg_direct_solve(self.h, _ptr(u), _ptr(f), _stream(stream)), "mg_direct_solve")
        return u

    # ---- cycles and solves
    def vcycle(self, u, f, params: Params | None = None, stream=None, **kw):
        p = params or default_params(**kw)
        _check(self.lib.mg_vcycle(self.h, _ptr(u), _ptr(f), ctypes.byref(p), _stream(stream)), "mg_vcycle")
        return u

    def _solve(self, fn, name, u, f, params, stream, history_cap, kw, raise_on_fail):
        p = params or default_params(**kw)
        hist = np.zeros(max(history_cap, 1))
        info = Info()
        info.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        info.history_cap = history_cap
        st = fn(self.h, _ptr(u), _ptr(f), ctypes.byref(p), ctypes.byref(info), _stream(stream))
        if raise_on_fail:
            _check(st, name)
        else:
            _check(st, name, ok=(OK, ERR_NOT_CONVERGED, ERR_NONFINITE))
        return SolveResult(st, info.cycles, info.outer_iters, info.rel_res, info.conv_factor, info.ms,
                           hist[: info.history_len].copy())

    def solve(self, u, f, params: Params | None = None, stream=None, history_cap=256, raise_on_fail=False, **kw):
        """mg_solve: u (float64 CUDA tensor, boundary values set; the solution on
        return), f (float64); params or default_params(**kw).  Returns a
        SolveResult with the status, cycles, residual history and convergence
        factor; raises MGError on a status other than OK / NOT_CONVERGED /
        NONFINITE (and on those too with raise_on_fail)."""
        return self._solve(self.lib.mg_solve, "mg_solve", u, f, params, stream, history_cap, kw, raise_on_fail)

    def solve_adjoint(self, lam, rhs, params: Params | None = None, stream=None, history_cap=256,
                      raise_on_fail=False, **kw):
        return self._solve(self.lib.mg_solve_adjoint, "mg_solve_adjoint", lam, rhs, params, stream, history_cap,
                           kw, raise_on_fail)


class Batch:
    """mg_batch_create over distinct Grid objects (which must outlive it)."""

    def __init__(self, grids):
        self.lib = load()
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(self.lib.mg_batch_create(ctypes.byref(h), len(self.grids), arr), "mg_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.mg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, us, fs, params=None, stream=None, history_cap=256, raise_on_fail=False, **kw) -> list:
        """mg_batch_solve: us[i], fs[i] float64 CUDA tensors of grid i; params:
        one Params for all problems, a list of one per problem, or None (the
        keyword arguments for all)."""
        n = len(self.grids)
        if len(us) != n or len(fs) != n:
            raise ValueError("one u and one f per grid")
        if isinstance(params, (list, tuple)):
            if len(params) != n:
                raise ValueError("one Params per grid")
            pa = (Params * n)(*params)
        else:
            pa = (Params * 1)(params or default_params(**kw))
        hists = [np.zeros(max(history_cap, 1)) for _ in range(n)]
        infos = (Info * n)()
        for i in range(n):
            infos[i].history = hists[i].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            infos[i].history_cap = history_cap
        ua = (ctypes.c_void_p * n)(*[_ptr(x).value for x in us])
        fa = (ctypes.c_void_p * n)(*[_ptr(x).value for x in fs])
        sts = (ctypes.c_int * n)()
        st = self.lib.mg_batch_solve(self.h, ua, fa, pa, len(pa), infos, sts, _stream(stream))
        if raise_on_fail:
            _check(st, "mg_batch_solve")
        else:
            _check(st, "mg_batch_solve", ok=(OK, ERR_NOT_CONVERGED, ERR_NONFINITE))
        return [SolveResult(int(sts[i]), infos[i].cycles, infos[i].outer_iters, infos[i].rel_res, infos[i].conv_factor,
                            infos[i].ms, hists[i][: infos[i].history_len].copy()) for i in range(n)]
