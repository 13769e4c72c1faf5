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


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    exe = tmp_path_factory.mktemp("p3d") / "pack3_dump"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "pack3_dump.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _read_lists(dumper, dims, smoother, colour):
    toks = subprocess.run([dumper], input=f"{dims[0]} {dims[1]} {dims[2]} {smoother} {colour}\n",
                          capture_output=True, text=True, check=True).stdout.split()
    it = iter(int(t) for t in toks)
    nwarp, K, W, nj, nskel = (next(it) for _ in range(5))
    cap = 32 * W * K
    slots = [[(next(it), next(it)) for _ in range(cap)] for _ in range(nwarp)]
    jofs = [next(it) for _ in range(nwarp + 1)]
    juncs = [(next(it), next(it), next(it), [next(it) for _ in range(6)]) for _ in range(nj)]
    skels = []
    for _ in range(nskel):
        c = [next(it) for _ in range(8)]
        eoff = [next(it) for _ in range(13)]
        ea = [next(it) for _ in range(12)]
        eb = [next(it) for _ in range(12)]
        ed = [next(it) for _ in range(12)]
        skels.append((c, eoff, ea, eb, ed))
    return slots, jofs, juncs, skels


@pytest.mark.parametrize("smoother", ["tweed", "wireframe"])
@pytest.mark.parametrize("dims", [(8, 8, 8), (16, 12, 10)])
def test_warp_lists_encode_the_block_systems(dumper, dims, smoother):
    """Assembling, from the descriptors alone, the linear system the 3D
    kernels solve (each slot's row with its predecessor, successor and
    junction couplings, every other neighbour on the right-hand side; the
    junction rows; the skeletons' edge and corner rows), and solving it
    densely, gives the oracle's colour pass."""
    import numpy as np
    import oracle
    from paper_2110_08389_gb300 import inputs as I

    nx, ny, nz = dims
    xyz = [I.coords(n, "wall" if smoother == "tweed" else "centre", ratio=20.0) for n in dims]
    P = oracle.Problem3(*xyz)
    co = P.coeffs()
    nx1, plane = nx + 1, (nx + 1) * (ny + 1)
    step = [1, -1, nx1, -nx1, plane, -plane]
    rng = np.random.default_rng(31)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())
    uf, ff = u0.ravel(), f.ravel()

    def pos(ijk):
        return (ijk >> 20) * plane + ((ijk >> 10) & 1023) * nx1 + (ijk & 1023)

    def ijk_of(p):
        return p % nx1, (p // nx1) % (ny + 1), p // plane

    def cdir(p, d):
        i, j, k = ijk_of(p)
        return [co["E"][i], co["W"][i], co["N"][j], co["S"][j], co["T"][k], co["B"][k]][d]

    for colour in (0, 1):
        ref = P.colour_pass(u0.copy(), f, colour, smoother=smoother).ravel()
        got = uf.copy()
        slots, jofs, juncs, skels = _read_lists(dumper, dims, {"tweed": 0, "wireframe": 1}[smoother], colour)
        multi = smoother == "wireframe"
        for w, seq in enumerate(slots):
            j0, nj = (jofs[w], jofs[w + 1] - jofs[w]) if multi else (w, 1)
            valid = [s for s, (_, fl) in enumerate(seq) if fl & (1 << 12)]
            if not valid:
                continue
            index = {s: r for r, s in enumerate(valid)}
            jrow = {e: len(valid) + r for r, e in enumerate(range(nj)) if juncs[j0 + e][1] > 0}
            n = len(valid) + len(jrow)
            A = np.zeros((n, n))
            b = np.zeros(n)
            for s in valid:
                ijk, fl = seq[s]
                p, r = pos(ijk), index[s]
                pd = fl & 7 if fl & (1 << 3) else None
                sd = (fl >> 4) & 7 if fl & (1 << 7) else None
                jd = (fl >> 8) & 7 if fl & (1 << 11) else None
                b[r] = ff[p]
                for d in range(6):
                    c = cdir(p, d)
                    A[r, r] -= c
                    if d == pd:
                        A[r, index[s - 1]] += c
                    elif d == sd:
                        A[r, index[s + 1]] += c
                    elif d == jd:
                        A[r, jrow[(fl >> 16) & 31]] += c
                    else:
                        b[r] -= c * uf[p + step[d]]
            for e, r in jrow.items():
                ijk, natt, adirs, att = juncs[j0 + e]
                p = pos(ijk)
                dirs = {(adirs >> (3 * a)) & 7: att[a] for a in range(natt)}
                b[r] = ff[p]
                for d in range(6):
                    c = cdir(p, d)
                    A[r, r] -= c
                    if d in dirs:
                        A[r, index[dirs[d]]] += c
                    else:
                        b[r] -= c * uf[p + step[d]]
            x = np.linalg.solve(A, b)
            for s in valid:
                got[pos(seq[s][0])] = x[index[s]]
            for e, r in jrow.items():
                got[pos(juncs[j0 + e][0])] = x[r]
        for c8, eoff, ea, eb, ed in skels:
            nodes = [pos(v) for v in c8]
            for e in range(12):
                for q in range(eoff[e + 1] - eoff[e]):
                    nodes.append(nodes[ea[e]] + (q + 1) * step[ed[e]])
            idx = {p: r for r, p in enumerate(nodes)}
            A = np.zeros((len(nodes), len(nodes)))
            b = np.zeros(len(nodes))
            for p, r in idx.items():
                b[r] = ff[p]
                for d in range(6):
                    c = cdir(p, d)
                    A[r, r] -= c
                    q = p + step[d]
                    if q in idx:
                        A[r, idx[q]] += c
                    else:
                        b[r] -= c * uf[q]
            x = np.linalg.solve(A, b)
            for p, r in idx.items():
                got[p] = x[r]
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (colour, np.abs(got - ref).max())
