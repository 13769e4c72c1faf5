"""The closed-form 2D block builders the GPU work lists are made from
(csrc/blocks.h), on the CPU: for every line smoother and colour their blocks
are exactly the oracle's blocks of that colour (the oracle finds them as
level sets of the wall distances, an independent construction), every chain
is a path of adjacent nodes and every junction link points at the junction."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
CODES = {"zebra_x": 0, "zebra_y": 1, "tweed": 2, "wireframe": 3}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = tmp_path_factory.mktemp("b2") / "blocks2_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "blocks2_driver.cpp"), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("smoother", list(CODES))
@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 16), (32, 16), (12, 40), (64, 64), (6, 10)])
def test_builder_blocks_are_the_oracle_blocks(driver, nx, ny, smoother):
    P = oracle.Problem(I.uniform_coords(nx), I.uniform_coords(ny))
    ref = P.owner(smoother)
    info = P.partition(smoother)  # (type, colour, size, legs) per block
    interior = np.zeros(ref.shape, dtype=bool)
    interior[1:-1, 1:-1] = True
    for colour in (0, 1):
        out = subprocess.run([driver], input=f"{nx} {ny} {CODES[smoother]} {colour}\n", capture_output=True,
                             text=True, check=True).stdout.split()
        got = np.array([int(v) for v in out[:-1]]).reshape(ny + 1, nx + 1)
        assert out[-1] == "1"
        mine = interior & (ref >= 0) & (info[np.maximum(ref, 0), 1] == colour)
        assert ((got >= 0) == mine).all(), (colour, np.argwhere((got >= 0) != mine)[:5])
        pairs = set(zip(got[mine].tolist(), ref[mine].tolist()))
        assert len(pairs) == len(set(got[mine].tolist())) == len(set(ref[mine].tolist()))
