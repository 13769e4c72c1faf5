"""Host part of the 3D tiled tweed path (csrc/tile3_host.h), on the CPU.

For each colour the layout is read back (tests/tile3_dump.cpp): every block
record's legs, through their chunks' lane slots (each the tile's run base
and direction, the lane's fixed coordinates and active slots), must be
straight chains of adjacent nodes whose first node follows a node outside
the block, ending at the junction (TL_LAST_J) or before a node outside the
block (TL_LAST_W); every used lane belongs to exactly one chunk.  The system
assembled from that layout alone (each node's row of Eq. (prob:DP) with the
block's nodes unknown and every other neighbour known), solved densely, must
give the oracle's 3D tweed colour pass (Sec. 7) at every
node: a node the layout lost, doubled, misplaced or coupled wrongly fails
it."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
STEP = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    exe = tmp_path_factory.mktemp("t3") / "tile3_dump"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "tile3_dump.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _layout(dumper, nx, ny, nz, colour):
    toks = subprocess.run([dumper], input=f"{nx} {ny} {nz} {colour}\n", capture_output=True, text=True,
                          check=True).stdout.split()
    assert toks[0] == "ok", toks[:2]
    it = iter(int(t) for t in toks[1:])
    nt, nb, ng, ns = next(it), next(it), next(it), next(it)
    tiles = [(next(it), next(it)) for _ in range(nt)]
    lanes = [tuple(next(it) for _ in range(4)) for _ in range(32 * nt)]
    blocks = [tuple(next(it) for _ in range(18)) for _ in range(nb)]
    slots = [next(it) for _ in range(ns)]
    assert nb == 32 * ng
    return tiles, lanes, blocks, slots


def _node(d, v, c1, c2):
    """(i, j, k) of run coordinate v on the run along direction d."""
    if d < 2:
        return v, c1, c2
    if d < 4:
        return c1, v, c2
    return c1, c2, v


@pytest.mark.parametrize("dims,kind", [((16, 16, 16), "wall"), ((24, 16, 32), "centre"), ((32, 32, 32), "wall"),
                                       ((16, 40, 24), "wall")])
def test_tile3_layout_encodes_the_block_systems(dumper, dims, kind):
    nx, ny, nz = dims
    x, y, z = (I.coords(n, kind, ratio=30.0) for n in dims)
    P = oracle.Problem3(x, y, z)
    c = P.coeffs()
    rng = np.random.default_rng(61)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())

    def coef(i, j, k, d):  # coupling of (i, j, k) to its neighbour in direction d
        return [c["E"][i], c["W"][i], c["N"][j], c["S"][j], c["T"][k], c["B"][k]][d]

    for colour in (0, 1):
        tiles, lanes, blocks, slots = _layout(dumper, nx, ny, nz, colour)
        used = np.zeros(32 * len(tiles), dtype=int)
        ref = P.colour_pass(u0.copy(), f, colour)
        got = u0.copy()
        covered = np.zeros(u0.shape, dtype=int)
        for bd in blocks:
            ji, jj, jk, nleg, junc, jdirs = bd[:6]
            s0s, lens = bd[6:12], bd[12:18]
            if nleg == 0 and not junc:
                continue
            assert nleg <= 6
            nodes, ends = [], []
            for l in range(nleg):
                leg, last = [], None
                for r in range((lens[l] + 31) // 32):
                    sl = slots[s0s[l] + r]
                    used[sl] += 1
                    base, d = tiles[sl // 32]
                    c1, c2, q1, flags = lanes[sl]
                    step = -1 if d & 1 else 1
                    for q in range(q1):
                        leg.append(_node(d, base + q * step, c1, c2))
                    if r == 0:
                        assert flags & 1  # TL_FIRST
                    last = (flags, d)
                assert len(leg) == lens[l] and len(leg) > 0
                d = last[1]
                for a, b in zip(leg, leg[1:]):
                    assert tuple(np.subtract(b, a)) == STEP[d]
                if junc:
                    assert last[0] & 2  # TL_LAST_J: the junction follows the last node
                    assert tuple(np.subtract((ji, jj, jk), leg[-1])) == STEP[d]
                    assert (jdirs >> (3 * l)) & 7 == d ^ 1
                else:
                    assert last[0] & 4  # TL_LAST_W
                nodes += leg
                ends.append((leg, d, junc))
            if junc:
                nodes.append((ji, jj, jk))
            idx = {p: n for n, p in enumerate(nodes)}
            assert len(idx) == len(nodes)
            for leg, d, jn in ends:  # the node before a leg, and after a free end, is outside the block
                assert tuple(np.subtract(leg[0], STEP[d])) not in idx
                if not jn:
                    assert tuple(np.add(leg[-1], STEP[d])) not in idx
            # the block's rows, assembled from the layout alone
            n = len(nodes)
            A, rhs = np.zeros((n, n)), np.zeros(n)
            for r, (i, j, k) in enumerate(nodes):
                covered[k, j, i] += 1
                A[r, r] = -sum(coef(i, j, k, d) for d in range(6))
                rhs[r] = f[k, j, i]
                for d in range(6):
                    q = (i + STEP[d][0], j + STEP[d][1], k + STEP[d][2])
                    if q in idx:
                        A[r, idx[q]] += coef(i, j, k, d)
                    else:
                        rhs[r] -= coef(i, j, k, d) * u0[q[2], q[1], q[0]]
            sol = np.linalg.solve(A, rhs)
            for (i, j, k), v in zip(nodes, sol):
                got[k, j, i] = v
        assert covered.max() == 1
        # every lane with slots belongs to exactly one leg's chunk
        assert np.array_equal(used > 0, np.array([ln[2] > 0 for ln in lanes])) and used.max() == 1
        changed = ref != u0
        assert np.all(covered[changed] == 1)
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-9 * scale
