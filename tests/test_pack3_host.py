"""Host part of the 3D warp lists (csrc/pack3_host.h), on the CPU: the
sequences hold every chain node of the colour exactly once, chains run
through consecutive slots with predecessor and successor directions that
point at the neighbouring slot's node, every junction record points back at
the slots attached to it, unused slots are zero, and the skeleton
descriptors' scratch offsets are consecutive."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = tmp_path_factory.mktemp("p3") / "pack3_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "pack3_driver.cpp"), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("colour", [0, 1])
@pytest.mark.parametrize("dims", [(8, 8, 8), (16, 12, 10), (24, 16, 32), (64, 48, 32)])
def test_warp_list_layout(driver, dims, smoother, colour):
    out = subprocess.run([driver], input=f"{dims[0]} {dims[1]} {dims[2]} {smoother} {colour}\n", capture_output=True,
                         text=True, check=True).stdout.split()
    assert out[0] == "ok", out
    nwarp, K, W, valid, nskel = (int(v) for v in out[1:])
    assert K in (1, 2, 4, 8) and W in (1, 2, 4, 8)
    assert valid > 0 and valid <= nwarp * 32 * W * K
    if smoother == 0:
        assert nskel == 0
