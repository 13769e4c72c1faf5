"""The C ABI library builds, loads without a GPU and exports every entry
point include/mg.h declares; host-only entry points behave."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_boundary():
    names = declared_functions()
    for required in ["mg_setup_grid", "mg_smooth_tweed", "mg_smooth_wireframe", "mg_vcycle", "mg_solve",
                     "mg_solve_adjoint", "mg_destroy", "mg_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2110_08389_gb300 import build, mg
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(mg.EXPORTS) == declared_functions()


def test_host_only_entry_points():
    from paper_2110_08389_gb300 import build, mg
    build.build()
    lib = mg.load()
    assert lib.mg_status_string(0) == b"ok"
    assert lib.mg_status_string(4) == b"not converged"
    p = mg.default_params()
    assert (p.smoother, p.nu1, p.nu2, p.cycle, p.restriction, p.tol) == (mg.TWEED, 2, 2, 1, mg.FW, 1e-10)
    assert lib.mg_num_levels(None) == 0
    assert lib.mg_solve(None, None, None, None, None, None) == mg.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.mg_setup_grid(ctypes.byref(h), 2, None, None, 3, None) == mg.ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: a missing CUDA library is an error, not a silent path."""
    import pytest
    from paper_2110_08389_gb300 import mg
    saved = mg._lib
    mg._lib = None
    try:
        with pytest.raises(RuntimeError):
            mg.load(str(tmp_path / "missing.so"))
    finally:
        mg._lib = saved


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the header's field offsets and sizes
    (checked by a small C program built with gcc against include/mg.h)."""
    import subprocess
    from paper_2110_08389_gb300 import mg
    structs = {"mg_params": mg.Params, "mg_info": mg.Info}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            c, k, v = line.split()
            got[(c, k)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_default_params():
    from paper_2110_08389_gb300 import mg
    p = mg.default_params()
    assert (p.smoother, p.nu1, p.nu2, p.inner_cycles, p.early_stop, p.coarse_direct) == (mg.TWEED, 2, 2, 3, 0, 0)


def test_checked_build_exports_and_reports_itself():
    """The checked variant (build.py --checked) exports the same entry points;
    mg_check_word needs no GPU in the plain build (returns 0)."""
    from paper_2110_08389_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.mg_check_word.restype = ctypes.c_uint
    assert lib.mg_check_word() == 0
    checked = ctypes.CDLL(build.build(checked=True))
    missing = [n for n in declared_functions() if not hasattr(checked, n)]
    assert not missing, missing
