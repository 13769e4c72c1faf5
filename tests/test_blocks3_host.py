"""Host part of the 3D block builder (csrc/blocks3_host.h), on the CPU: the
tweed and wireframe blocks it lays out for the GPU passes are exactly the
oracle's blocks (same node sets, same colours), every chain is a path of
adjacent nodes, every junction attachment and skeleton edge is where the
kernels will look for it, and every interior node is in one block."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = tmp_path_factory.mktemp("b3") / "blocks3_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "blocks3_driver.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def build_blocks(driver, nx, ny, nz, sm):
    out = subprocess.run([driver], input=f"{nx} {ny} {nz} {sm}\n", capture_output=True, text=True,
                         check=True).stdout.split()
    ok, nb = int(out[0]), int(out[1])
    assert ok == 1
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    owner = np.array([int(v) for v in out[2:2 + nn]]).reshape(nz + 1, ny + 1, nx + 1)
    colour = np.array([int(v) for v in out[2 + nn:2 + nn + nb]])
    shapes = int(out[2 + nn + nb])
    return owner, colour, shapes


@pytest.mark.parametrize("smoother", ["tweed", "wireframe"])
@pytest.mark.parametrize("dims", [(8, 8, 8), (16, 12, 10), (24, 16, 32), (12, 20, 6)])
def test_builder_blocks_are_the_oracle_blocks(driver, dims, smoother):
    nx, ny, nz = dims
    owner, colour, shapes = build_blocks(driver, nx, ny, nz, {"tweed": 0, "wireframe": 1}[smoother])
    assert shapes == 1
    P = oracle.Problem3(*(I.uniform_coords(n) for n in dims))
    ref_owner, ref_colour = P.partition(smoother=smoother)
    interior = np.zeros(owner.shape, dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    assert (owner[interior] >= 0).all() and (owner[~interior] == -1).all()
    # the same partition up to block numbering, with the same colours
    pairs = set(zip(owner[interior].tolist(), ref_owner[interior].tolist()))
    assert len(pairs) == len(set(owner[interior].tolist())) == len(set(ref_owner[interior].tolist()))
    for b, rb in pairs:
        assert colour[b] == ref_colour[rb]
