"""Host part of the cluster pass (csrc/cluster_host.h) and its chunk
arithmetic (csrc/cluster_math.h), on the CPU: a g++ driver runs one colour
pass the way the kernel's CTAs split it -- chunk right-hand sides and reduced
rows in each CTA's own arrays, each block's legs solved by the CTA the kernel
gives it (Thomas from the wall, the junction row, back-substitution) on rows
and end values held by the other CTAs of its cluster, chunk recovery -- in
FP64; every chunk's end values must be written exactly once, and the result
must equal the oracle's colour pass of tweed and zebra (Sec. 3) to rounding.
Small tile and cluster sizes make the groups of small grids span several
CTAs, as the large levels' groups do."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
WL = {"zebra_x": 0, "zebra_y": 1, "tweed": 2}


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    exe = tmp_path_factory.mktemp("cl") / "cluster_emulate"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "cluster_emulate.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _run(emulator, P, u, f, wl, colour, S, CL):
    ny1, nx1 = P.shape()
    W, E, Sc, N = P.coeffs()
    parts = [f"{nx1 - 1} {ny1 - 1} {wl} {colour} {S} {CL}"]
    for a in (W, E, Sc, N, u.ravel(), f.ravel()):
        parts.append(" ".join(repr(float(v)) for v in a))
    r = subprocess.run([emulator], input="\n".join(parts) + "\n", capture_output=True, text=True)
    assert r.returncode == 0, r.returncode
    out = r.stdout.split("\n")
    if out[0] == "noplan":
        return None, None
    head = [int(v) for v in out[0].split()[1:]]
    return head, np.array([float(v) for v in out[1:1 + ny1 * nx1]]).reshape(ny1, nx1)


@pytest.mark.parametrize("smoother", list(WL))
@pytest.mark.parametrize("nx,ny,kind,S,CL", [
    (64, 64, "wall", 2, 4),       # L-blocks over up to 4 CTAs, the cross compact
    (64, 64, "wall", 1, 8),       # one tile per CTA
    (128, 64, "wall", 2, 8),      # T-blocks (compact) and wall-to-wall lines
    (64, 160, "centre", 4, 8),
    (96, 96, "centre", 16, 8),    # the kernel's own sizes: every group in one CTA
    (200, 200, "wall", 3, 8),     # ragged chunks and uneven CTA splits
])
def test_cluster_pass_equals_oracle(emulator, nx, ny, kind, S, CL, smoother):
    x, y = I.coords(nx, kind, ratio=50.0), I.coords(ny, kind, ratio=50.0)
    P = oracle.Problem(x, y)
    rng = np.random.default_rng(61)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())
    for colour in (0, 1):
        ref = P.colour_pass(u0.copy(), f, smoother, colour)
        head, got = _run(emulator, P, u0, f, WL[smoother], colour, S, CL)
        assert head is not None, "no plan"
        ncta = head[0]
        assert ncta % CL == 0
        changed = ref != u0
        assert np.array_equal(got[~changed], u0[~changed])  # the other colour and the boundary untouched
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (colour, np.abs(got - ref).max())


def test_cluster_plan_sizes(emulator):
    """The default plan (16 tiles per CTA, clusters of 8) exists for the
    4097^2 and 2049^2 levels of tweed and both zebras, and a group that needs
    more CTAs than a cluster holds gives no plan (the tiled path is used)."""
    P = oracle.Problem(I.uniform_coords(64), I.uniform_coords(64))
    u0 = np.zeros(P.shape())
    # 64 intervals: a zebra line is 63 nodes = 2 chunks; 1 tile per CTA, 1 CTA per cluster: no plan
    head, _ = _run(emulator, P, u0, u0, 0, 0, 1, 1)
    assert head is None
    drv = os.path.join(os.path.dirname(emulator), "cluster_plan_stats")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "cluster_plan_stats.cpp"), "-o", drv], check=True)
    for n in (2048, 4096):
        for wl in (0, 1, 2):
            totals = 0
            for colour in (0, 1):
                out = subprocess.run([drv], input=f"{n} {n} {wl} {colour}\n", capture_output=True, text=True,
                                     check=True).stdout.split()
                ok, ncta, ntile, nodes, junc, total, max_seg, idle = (int(v) for v in out)
                assert ok == 1 and ncta % 8 == 0 and ntile > 0
                assert nodes + junc == total  # every unknown in one chunk slot or a junction
                assert max_seg <= 128
                assert idle <= ncta // 8  # the packing leaves few CTAs idle
                totals += total
            assert totals == (n - 1) ** 2
