"""Host part of the tiled line path (csrc/tile_host.h), on the CPU: each
block record's legs, read through its tiles and lane (run base and
direction, the lane's fixed coordinate and active slots), are chains of
adjacent nodes that start at a wall and end at the junction or the other
wall; the system assembled from that layout and solved densely gives the
oracle's tweed and zebra colour passes."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
WL = {"zebra_x": 0, "zebra_y": 1, "tweed": 2}
DI, DJ = [1, -1, 0, 0], [0, 0, 1, -1]


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    exe = tmp_path_factory.mktemp("tl") / "tile_dump"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "tile_dump.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _layout(dumper, nx, ny, wl, colour):
    toks = subprocess.run([dumper], input=f"{nx} {ny} {wl} {colour}\n", capture_output=True, text=True,
                          check=True).stdout.split()
    it = iter(int(t) for t in toks)
    nt, nb = next(it), next(it)
    tiles = [(next(it), next(it)) for _ in range(nt)]
    lanes = [tuple(next(it) for _ in range(4)) for _ in range(32 * nt)]
    blocks = [tuple(next(it) for _ in range(14)) for _ in range(nb)]
    return tiles, lanes, blocks


@pytest.mark.parametrize("smoother", list(WL))
@pytest.mark.parametrize("nx,ny,kind", [(64, 64, "wall"), (128, 64, "wall"), (64, 160, "centre"), (96, 96, "centre")])
def test_tile_layout_encodes_the_block_systems(dumper, nx, ny, kind, smoother):
    x, y = I.coords(nx, kind, ratio=50.0), I.coords(ny, kind, ratio=50.0)
    P = oracle.Problem(x, y)
    cW, cE, cS, cN = P.coeffs()
    rng = np.random.default_rng(51)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())

    def coef(i, j, d):
        return [cE[i], cW[i], cN[j], cS[j]][d]

    def wall(i, j):
        return i == 0 or i == nx or j == 0 or j == ny

    for colour in (0, 1):
        tiles, lanes, blocks = _layout(dumper, nx, ny, WL[smoother], colour)
        ref = P.colour_pass(u0.copy(), f, smoother, colour)
        got = u0.copy()
        covered = np.zeros(u0.shape, dtype=int)
        for bd in blocks:
            ji, jj, nleg, junc, jdirs, lane = bd[:6]
            t0s, lens = bd[6:10], bd[10:14]
            if nleg == 0 and not junc:
                continue
            nodes, links = [], set()
            ends = []
            for l in range(nleg):
                leg = []
                for r in range((lens[l] + 31) // 32):
                    base, d = tiles[t0s[l] + r]
                    line, q0, q1, flags = lanes[32 * (t0s[l] + r) + lane]
                    step = 1 if d in (0, 2) else -1
                    for q in range(q0, q1):
                        v = base + q * step
                        p = (v, line) if d < 2 else (line, v)
                        if not leg and flags & 1:  # the first node's predecessor is a wall node
                            assert wall(p[0] - DI[d], p[1] - DJ[d])
                        leg.append(p)
                    last_flags, last_dir = flags, d
                assert len(leg) == lens[l]
                # the leg's last lane says where the leg ends: the junction or a wall node
                if junc:
                    assert last_flags & 2
                else:
                    assert last_flags & 4 and wall(leg[-1][0] + DI[last_dir], leg[-1][1] + DJ[last_dir])
                for a, b in zip(leg, leg[1:]):
                    assert abs(a[0] - b[0]) + abs(a[1] - b[1]) == 1
                    links.add((a, b))
                    links.add((b, a))
                nodes += leg
                ends.append((leg[-1], (jdirs >> (2 * l)) & 3))
            if junc:
                J = (ji, jj)
                for e, dj in ends:
                    assert (J[0] + DI[dj], J[1] + DJ[dj]) == e
                    links.add((e, J))
                    links.add((J, e))
                nodes.append(J)
            idx = {p: r for r, p in enumerate(nodes)}
            assert len(idx) == len(nodes)
            A = np.zeros((len(nodes), len(nodes)))
            b = np.zeros(len(nodes))
            for p, r in idx.items():
                i, j = p
                covered[j, i] += 1
                b[r] = f[j, i]
                for d in range(4):
                    c = coef(i, j, d)
                    A[r, r] -= c
                    q = (i + DI[d], j + DJ[d])
                    if (p, q) in links:
                        A[r, idx[q]] += c
                    else:
                        b[r] -= c * u0[q[1], q[0]]
            xs = np.linalg.solve(A, b)
            for p, r in idx.items():
                got[p[1], p[0]] = xs[r]
        assert covered.max() <= 1 and (covered[ref != u0] == 1).all()
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (colour, np.abs(got - ref).max())


@pytest.mark.parametrize("smoother", list(WL))
@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 64), (64, 160), (96, 96), (256, 128)])
def test_wide_blocks_alone_in_their_group(dumper, nx, ny, smoother):
    """The FP32 couple with precomputed pivots gives every leg of a group one
    of 64 shared-memory slots: legs 0 and 1 of the group's 32 blocks, and legs
    2 and 3 only of a block alone in its group.  So a block of three or four
    legs (the centre cross, the T-blocks) must sit at lane 0 of a group whose
    other 31 records are empty; the setup checks the same (pc_slots_ok) and
    keeps the plain couple otherwise."""
    for colour in (0, 1):
        _, _, blocks = _layout(dumper, nx, ny, WL[smoother], colour)
        assert len(blocks) % 32 == 0
        for g0 in range(0, len(blocks), 32):
            grp = blocks[g0:g0 + 32]
            for q, bd in enumerate(grp):
                ji, jj, nleg, junc, jdirs, lane = bd[:6]
                assert nleg <= 4
                if nleg > 2:
                    assert q == 0 and lane == 0
                    assert all(o[2] == 0 and o[3] == 0 for o in grp[1:])
