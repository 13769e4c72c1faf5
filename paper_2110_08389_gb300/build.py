"""Build the tweedmg CUDA library in-tree for sm_103a.

``python -m paper_2110_08389_gb300.build`` (or :func:`build`) compiles every
``csrc/*.cu`` translation unit with nvcc in parallel and links
``_build/libtweedmg.so``.  Rebuilds only when a source or header is newer
than the library.

``build(checked=True)`` (``--checked``) builds the checked variant into
``_build_check/libtweedmg.so``: compiled with ``-DMG_CHECK``, its kernels
validate the indices they decode from their descriptors and record any that
is out of range (see csrc/device_util.cuh); mg.py loads it when the
environment variable TWEEDMG_LIB names it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtweedmg.so")
OUT_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(OUT_CHECK, "libtweedmg.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", f"-I{INCLUDE}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the tweedmg CUDA library cannot be built")


def _stale(srcs, target) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = srcs + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    out, lib = (OUT_CHECK, LIB_CHECK) if checked else (OUT, LIB)
    if not force and not _stale(srcs, lib):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + (["-DMG_CHECK"] if checked else []) + (extra or [])

    def compile_one(src):
        obj = os.path.join(out, os.path.basename(src) + ".o")
        tu = [f'-DMG_CHECK_TU="{os.path.basename(src)}"'] if checked else []
        cmd = [cc, *ARCH, *flags, *tu, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None, checked="--checked" in sys.argv))
