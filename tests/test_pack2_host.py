"""Host part of the 2D warp lists (csrc/pack2_host.h), on the CPU: the system
assembled from the descriptors alone -- each slot's row with its
predecessor, successor and junction couplings, every other neighbour on the
right-hand side, and each sequence's junction row -- solved densely, gives
the oracle's colour pass for zebra x/y, tweed and wireframe."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
CODES = {"zebra_x": 0, "zebra_y": 1, "tweed": 2, "wireframe": 3}
DI, DJ = [1, -1, 0, 0], [0, 0, 1, -1]


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    exe = tmp_path_factory.mktemp("p2") / "pack2_dump"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "pack2_dump.cpp"), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("smoother", list(CODES))
@pytest.mark.parametrize("nx,ny,kind", [(16, 16, "wall"), (32, 16, "centre"), (12, 40, "wall"), (64, 64, "centre")])
def test_warp_list_encodes_the_block_systems(dumper, nx, ny, kind, smoother):
    x, y = I.coords(nx, kind, ratio=30.0), I.coords(ny, kind, ratio=30.0)
    P = oracle.Problem(x, y)
    cW, cE, cS, cN = P.coeffs()
    rng = np.random.default_rng(41)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())
    nx1 = nx + 1

    def coef(i, j, d):
        return [cE[i], cW[i], cN[j], cS[j]][d]

    for colour in (0, 1):
        out = subprocess.run([dumper], input=f"{nx} {ny} {CODES[smoother]} {colour} 16 4\n", capture_output=True,
                             text=True, check=True).stdout.split()
        assert out[0] == "ok"
        it = iter(int(t) for t in out[1:])
        nwarp, K, W = next(it), next(it), next(it)
        cap = 32 * W * K
        slots = [[(next(it), next(it), next(it)) for _ in range(cap)] for _ in range(nwarp)]
        blks = [[next(it) for _ in range(9)] for _ in range(nwarp)]
        ref = P.colour_pass(u0.copy(), f, smoother, colour)
        got = u0.copy()
        covered = np.zeros(u0.shape, dtype=int)
        for seq, jb in zip(slots, blks):
            valid = [s for s, (_, _, fl) in enumerate(seq) if fl & (1 << 9)]
            has_j, ji, jj, natt, adirs = jb[:5]
            att = jb[5:]
            index = {s: r for r, s in enumerate(valid)}
            n = len(valid) + (1 if has_j else 0)
            A = np.zeros((n, n))
            b = np.zeros(n)
            for s in valid:
                i, j, fl = seq[s]
                r = index[s]
                covered[j, i] += 1
                pd = fl & 3 if fl & (1 << 2) else None
                sd = (fl >> 3) & 3 if fl & (1 << 5) else None
                jd = (fl >> 6) & 3 if fl & (1 << 8) else None
                b[r] = f[j, i]
                for d in range(4):
                    c = coef(i, j, d)
                    A[r, r] -= c
                    if d == pd:
                        A[r, index[s - 1]] += c
                    elif d == sd:
                        A[r, index[s + 1]] += c
                    elif d == jd:
                        A[r, n - 1] += c
                    else:
                        b[r] -= c * u0[j + DJ[d], i + DI[d]]
            if has_j:
                covered[jj, ji] += 1
                dirs = {(adirs >> (2 * e)) & 3: att[e] for e in range(natt)}
                r = n - 1
                b[r] = f[jj, ji]
                for d in range(4):
                    c = coef(ji, jj, d)
                    A[r, r] -= c
                    if d in dirs:
                        A[r, index[dirs[d]]] += c
                    else:
                        b[r] -= c * u0[jj + DJ[d], ji + DI[d]]
            if n == 0:
                continue
            xs = np.linalg.solve(A, b)
            for s in valid:
                i, j, _ = seq[s]
                got[j, i] = xs[index[s]]
            if has_j:
                got[jj, ji] = xs[n - 1]
        changed = ref != u0
        assert (covered[changed] == 1).all() and covered.max() <= 1
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (colour, np.abs(got - ref).max())
