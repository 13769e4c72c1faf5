"""Pins of the 3D tweed and wireframe oracle (oracle/mg_oracle3d.c, Sec. 7)
against what the paper and the mathematics fix: block shapes the paper
describes, the disjointness of the two motifs and their complement (Sec. 7,
complementarity), exact block solves against a dense library solve, the
properties of the 7-point operator, the tensor-product transfers, and the
multigrid solve against a dense LU solve and against a manufactured solution
(second-order convergence)."""
import numpy as np
import pytest

import oracle
from paper_2110_08389_gb300 import inputs as I

DIRS = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


def grid3(nx, ny, nz, kind="wall", ratio=20.0):
    if kind == "uniform":
        return I.uniform_coords(nx), I.uniform_coords(ny), I.uniform_coords(nz)
    return I.coords(nx, kind, ratio=ratio), I.coords(ny, kind, ratio=ratio), I.coords(nz, kind, ratio=ratio)


def interior_nodes(shape):
    nz1, ny1, nx1 = shape
    for k in range(1, nz1 - 1):
        for j in range(1, ny1 - 1):
            for i in range(1, nx1 - 1):
                yield k, j, i


def in_block_degree(owner, k, j, i):
    b = owner[k, j, i]
    return sum(1 for dk, dj, di in [(d[2], d[1], d[0]) for d in DIRS] if owner[k + dk, j + dj, i + di] == b)


@pytest.mark.parametrize("dims", [(8, 8, 8), (10, 8, 6), (12, 12, 12), (9, 7, 11)])
def test_partition_is_a_proper_block_colouring_of_stars(dims):
    P = oracle.Problem3(*grid3(*dims))
    owner, colour = P.partition()
    nz1, ny1, nx1 = owner.shape
    interior = np.zeros_like(owner, dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    assert (owner[interior] >= 0).all() and (owner[~interior] == -1).all()
    nb = len(colour)
    sizes = np.bincount(owner[interior], minlength=nb)
    assert (sizes > 0).all()
    edges = np.zeros(nb, dtype=np.int64)
    for k, j, i in interior_nodes(owner.shape):
        for di, dj, dk in DIRS[1::2]:  # +x, +y, +z once per edge
            kk, jj, ii = k + dk, j + dj, i + di
            if not interior[kk, jj, ii]:
                continue
            a, b = owner[k, j, i], owner[kk, jj, ii]
            if a == b:
                edges[a] += 1
            else:
                # neighbouring blocks always have different colours
                assert colour[a] != colour[b], ((k, j, i), (kk, jj, ii))
    nx, ny, nz = nx1 - 1, ny1 - 1, nz1 - 1
    if nx % 2 == 0 and ny % 2 == 0 and nz % 2 == 0:
        # every block is a tree (connected by construction: edges = nodes - 1)
        assert (edges == sizes - 1).all()
        # ... and a star: at most one node with three or more in-block neighbours
        branch = np.zeros(nb, dtype=np.int64)
        for k, j, i in interior_nodes(owner.shape):
            if in_block_degree(owner, k, j, i) >= 3:
                branch[owner[k, j, i]] += 1
        assert (branch <= 1).all()
    else:
        # an odd side has two middle lines at the same wall distance: their
        # blocks close loops (solved densely by the oracle)
        assert (edges >= sizes - 1).all() and (edges > sizes - 1).any()
    # the eight corner points are single-node red blocks (Sec. 7: "first relaxed")
    for i in (1, nx - 1):
        for j in (1, ny - 1):
            for k in (1, nz - 1):
                b = owner[k, j, i]
                assert sizes[b] == 1 and colour[b] == 0


@pytest.mark.parametrize("n", [8, 12])
def test_cube_centre_block_has_six_legs(n):
    """Sec. 7: with nx = ny = nz a single m = 6 block arises at the centre."""
    P = oracle.Problem3(*grid3(n, n, n))
    owner, colour = P.partition()
    c = n // 2
    assert in_block_degree(owner, c, c, c) == 6
    b = owner[c, c, c]
    # its legs run from the centre to the six walls: 6 (c - 1) + 1 nodes
    assert (owner == b).sum() == 6 * (c - 1) + 1


@pytest.mark.parametrize("smoother", ["tweed", "wireframe", "complementary"])
@pytest.mark.parametrize("dims", [(8, 6, 10), (7, 6, 5)])
def test_block_solve_equals_dense_solve(dims, smoother):
    """Every block solve (tree elimination; dense for loops) equals numpy's
    dense solve of that block's system, the other nodes held fixed (Sec. 3:
    exact block relaxation)."""
    P = oracle.Problem3(*grid3(*dims, "wall", 50.0))
    rng = np.random.default_rng(3)
    shape = P.shape()
    u0, f = rng.standard_normal(shape), rng.standard_normal(shape)
    owner, colour = P.partition(smoother=smoother)
    co = P.coeffs()
    for b in range(len(colour)):
        nodes = [tuple(x) for x in np.argwhere(owner == b)]
        idx = {p: n for n, p in enumerate(nodes)}
        A = np.zeros((len(nodes), len(nodes)))
        r = np.zeros(len(nodes))
        for n, (k, j, i) in enumerate(nodes):
            c6 = [co["W"][i], co["E"][i], co["S"][j], co["N"][j], co["B"][k], co["T"][k]]
            A[n, n] = -sum(c6)
            r[n] = f[k, j, i]
            for d, (di, dj, dk) in enumerate(DIRS):
                q = (k + dk, j + dj, i + di)
                if q in idx:
                    A[n, idx[q]] = c6[d]
                else:
                    r[n] -= c6[d] * u0[q]
        x = np.linalg.solve(A, r)
        u = u0.copy()
        P.block_solve(b, u, f, smoother=smoother)
        got = np.array([u[p] for p in nodes])
        assert np.abs(got - x).max() <= 1e-12 * max(1.0, np.abs(x).max()), b
        mask = owner != b
        assert np.array_equal(u[mask], u0[mask])


@pytest.mark.parametrize("smoother", ["tweed", "wireframe", "complementary"])
def test_colour_pass_zeroes_the_relaxed_rows(smoother):
    P = oracle.Problem3(*grid3(12, 10, 8, "wall", 200.0))
    rng = np.random.default_rng(4)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())
    owner, colour = P.partition(smoother=smoother)
    for c in (0, 1):
        u = P.colour_pass(u0.copy(), f, c, smoother=smoother)
        d = P.residual(u, f)
        scale = np.abs(P.apply(np.abs(u)) * 0 + f).max() + np.abs(P.coeffs()["W"]).max() * np.abs(u).max() * 6
        relaxed = (owner >= 0) & (colour[np.maximum(owner, 0)] == c)
        assert np.abs(d[relaxed]).max() <= 1e-12 * scale
        assert np.array_equal(u[~relaxed], u0[~relaxed])


def test_operator_properties():
    """The 7-point operator: rows sum to zero (constant fields are in the
    kernel of L), D L is symmetric with D = diag(dx_i dy_j dz_k), and the
    uniform grid gives 1/h^2 coefficients."""
    x, y, z = grid3(6, 5, 4, "wall", 30.0)
    P = oracle.Problem3(x, y, z)
    shape = P.shape()
    assert np.abs(P.apply(np.ones(shape))).max() <= 1e-9 * np.abs(P.coeffs()["W"]).max()
    inner = [(k, j, i) for k, j, i in interior_nodes(shape)]
    n = len(inner)
    A = np.zeros((n, n))
    for c, p in enumerate(inner):
        e = np.zeros(shape)
        e[p] = 1.0
        Le = P.apply(e)
        A[:, c] = [Le[q] for q in inner]
    dx = lambda a, m: 0.5 * (a[m + 1] - a[m - 1])
    D = np.array([dx(x, i) * dx(y, j) * dx(z, k) for k, j, i in inner])
    DA = D[:, None] * A
    assert np.abs(DA - DA.T).max() <= 1e-12 * np.abs(DA).max()
    U = oracle.Problem3(*grid3(4, 4, 4, "uniform"))
    co = U.coeffs()
    for key in "WESNBT":
        assert np.allclose(co[key][1:-1], 16.0, rtol=1e-13)


def test_transfers_are_tensor_products():
    P = oracle.Problem3(*grid3(16, 16, 16, "wall", 10.0))
    # full weighting (weights 1/4, 1/2, 1/4 per axis) keeps a constant at
    # coarse nodes whose 27 fine neighbours are all interior
    d = np.zeros(P.shape(0))
    d[1:-1, 1:-1, 1:-1] = 3.0
    fc = P.restrict(d)
    assert np.allclose(fc[2:-2, 2:-2, 2:-2], 3.0, rtol=1e-14)
    # trilinear prolongation reproduces an index-linear coarse field exactly
    nzc, nyc, nxc = P.shape(1)
    K, J, Ic = np.meshgrid(np.arange(nzc), np.arange(nyc), np.arange(nxc), indexing="ij")
    uc = 1.0 + 2.0 * Ic - 3.0 * J + 0.5 * K
    u = P.prolong_add(uc, np.zeros(P.shape(0)))
    k, j, i = np.meshgrid(*[np.arange(s) for s in P.shape(0)], indexing="ij")
    ref = 1.0 + 2.0 * (i / 2) - 3.0 * (j / 2) + 0.5 * (k / 2)
    inner = (slice(1, -1),) * 3
    assert np.allclose(u[inner], ref[inner], rtol=0, atol=1e-12)


@pytest.mark.parametrize("smoother,kind,nz,ratio", [("tweed", "wall", 8, 100.0), ("wireframe", "centre", 16, 10.0)])
def test_multigrid_solve_equals_dense_lu(smoother, kind, nz, ratio):
    x, y, z = grid3(16, 16, nz, kind, ratio)
    P = oracle.Problem3(x, y, z)
    assert P.nlev == 2
    rng = np.random.default_rng(5)
    f = rng.standard_normal(P.shape())
    g = rng.standard_normal(P.shape())
    g[1:-1, 1:-1, 1:-1] = 0.0
    ref = P.direct_solve(g.copy(), f)
    u = g.copy()
    hist = P.solve(u, f, nu1=2, nu2=2, tol=1e-12, max_cycles=60, smoother=smoother)
    assert hist[-1] <= 1e-12 and len(hist) < 40
    assert np.abs(u - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["uniform", "wall"])
def test_second_order_convergence(kind):
    """u = sin(pi x) sin(pi y) sin(pi z) with f = -3 pi^2 u: the discrete
    solution's max error falls by about 4 when the grid is refined."""
    errs = []
    for n in (8, 16, 32):
        # a fixed mapping (fixed c), refined: the spacing halves everywhere
        x = I.uniform_coords(n) if kind == "uniform" else I.coords(n, "wall", c=1.5)
        y = z = x
        P = oracle.Problem3(x, y, z)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        ue = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        f = -3 * np.pi ** 2 * ue
        u = np.zeros(P.shape())
        P.solve(u, f, tol=1e-12, max_cycles=60)
        errs.append(np.abs(u - ue).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


def test_tweed_cycles_converge_on_stretched_grid():
    """3D tweed V(1,1) cycles on a grid stretched towards all six walls."""
    x, y, z = grid3(32, 32, 32, "wall", 200.0)
    P = oracle.Problem3(x, y, z)
    f = np.random.default_rng(6).standard_normal(P.shape())
    u = np.zeros(P.shape())
    hist = P.solve(u, f, nu1=1, nu2=1, tol=1e-10, max_cycles=40)
    assert hist[-1] <= 1e-10
    assert (hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1)) < 0.35


def block_graph(owner):
    """Per block: node count, in-block edge count, in-block degree of every
    interior node (a brute-force walk over the grid, independent of the
    oracle's construction)."""
    nb = owner.max() + 1
    sizes = np.bincount(owner[owner >= 0], minlength=nb)
    edges = np.zeros(nb, dtype=np.int64)
    deg = np.zeros(owner.shape, dtype=np.int64)
    for k, j, i in interior_nodes(owner.shape):
        for di, dj, dk in DIRS[1::2]:
            kk, jj, ii = k + dk, j + dj, i + di
            if owner[kk, jj, ii] >= 0 and owner[kk, jj, ii] == owner[k, j, i]:
                edges[owner[k, j, i]] += 1
                deg[k, j, i] += 1
                deg[kk, jj, ii] += 1
    return sizes, edges, deg


def classify(owner, b, sizes, edges, deg):
    d = deg[owner == b]
    n, e = sizes[b], edges[b]
    if n == 1:
        return "point"
    if e == n - 1 and d.max() <= 2:
        return "path"
    if e == n and (d == 2).all():
        return "ring"
    if e == n + 4 and (d == 3).sum() == 8 and (d[d != 3] == 2).all():
        return "skeleton"
    return "other"


@pytest.mark.parametrize("dims", [(10, 10, 10), (10, 8, 6), (16, 12, 10), (8, 8, 16)])
def test_wireframe_blocks_are_rings_on_cuboid_faces_and_edge_skeletons(dims):
    """Sec. 7: wireframe blocks cover the faces of concentric cuboids; on each
    cuboid the twelve edges form one block (eight three-way corners, a graph
    with five independent loops), and every face carries concentric rings
    (Eq. CircTri systems), closing in a line or a point at the face centre."""
    P = oracle.Problem3(*grid3(*dims, "centre", 20.0))
    owner, colour = P.partition(smoother="wireframe")
    sizes, edges, deg = block_graph(owner)
    kinds = [classify(owner, b, sizes, edges, deg) for b in range(len(colour))]
    assert "other" not in kinds
    nx, ny, nz = dims
    # one skeleton per concentric cuboid whose three sides are all at least 2
    n_skel = sum(1 for t in range(1, min(dims) // 2) if min(nx, ny, nz) - 2 * t >= 2)
    assert kinds.count("skeleton") == n_skel
    # the outermost skeleton (through the corner node (1, 1, 1)) is red: the
    # relaxation starts at the domain faces
    b0 = owner[1, 1, 1]
    assert kinds[b0] == "skeleton" and colour[b0] == 0
    # skeleton nodes are exactly the nodes whose two smallest wall distances
    # are equal (d1 == d2) on a cuboid with no flat side; on a flat cuboid
    # (its smallest side 0) those nodes close a ring, a line or a point
    for k, j, i in interior_nodes(owner.shape):
        a = sorted([min(i, nx - i), min(j, ny - j), min(k, nz - k)])
        solid = min(dims) - 2 * a[0] >= 2
        assert (kinds[owner[k, j, i]] == "skeleton") == (a[0] == a[1] and solid), (k, j, i)
    # neighbouring blocks differ in colour
    for k, j, i in interior_nodes(owner.shape):
        for di, dj, dk in DIRS[1::2]:
            kk, jj, ii = k + dk, j + dj, i + di
            a, b = owner[k, j, i], owner[kk, jj, ii]
            if b >= 0 and a != b:
                assert colour[a] != colour[b]


@pytest.mark.parametrize("n", [8, 12])
def test_wireframe_cube_has_point_blocks_at_face_centres(n):
    """Sec. 7: with nx = ny = nz a point relaxation sits at the centre of each
    face of each concentric cuboid."""
    P = oracle.Problem3(*grid3(n, n, n, "centre", 20.0))
    owner, _ = P.partition(smoother="wireframe")
    sizes = np.bincount(owner[owner >= 0])
    c = n // 2
    for t in range(1, c):
        for p in [(t, c, c), (n - t, c, c), (c, t, c), (c, n - t, c), (c, c, t), (c, c, n - t)]:
            if t < c:
                assert sizes[owner[p]] == 1, (t, p)


@pytest.mark.parametrize("dims", [(10, 10, 10), (12, 8, 6)])
def test_tweed_and_wireframe_are_disjoint_and_leave_the_complementary_wires(dims):
    """Sec. 7 (complementarity): the in-block wires of the tweed and wireframe
    motifs never overlap, and every wire left over connects two nodes that
    keep the smallest and largest of their three wall distances, the
    complementary wireframe motif that circles the cuboids' corners."""
    P = oracle.Problem3(*grid3(*dims))
    ot, _ = P.partition(smoother="tweed")
    ow, _ = P.partition(smoother="wireframe")
    nx, ny, nz = dims

    def srt(k, j, i):
        return sorted([min(i, nx - i), min(j, ny - j), min(k, nz - k)])

    counts = {"tweed": 0, "wireframe": 0, "rest": 0}
    for k, j, i in interior_nodes(ot.shape):
        for di, dj, dk in DIRS[1::2]:
            kk, jj, ii = k + dk, j + dj, i + di
            if ot[kk, jj, ii] < 0:
                continue
            in_t = ot[k, j, i] == ot[kk, jj, ii]
            in_w = ow[k, j, i] == ow[kk, jj, ii]
            assert not (in_t and in_w), (k, j, i)
            if in_t:
                counts["tweed"] += 1
            elif in_w:
                counts["wireframe"] += 1
            else:
                a, b = srt(k, j, i), srt(kk, jj, ii)
                assert a[0] == b[0] and a[2] == b[2] and a[1] != b[1]
                counts["rest"] += 1
    assert min(counts.values()) > 0


def test_wireframe_cycles_converge_on_centre_clustered_grid():
    """3D wireframe V(2,2) cycles on a grid clustered towards the centre
    (Eq. tanh_inv on every axis), the case wireframe is built for: faster
    than tweed there.  (Near the centre planes' intersections the cells are
    thin in two directions at once, which line blocks do not cover, so the
    rate stays well above the 2D one.)"""
    x, y, z = grid3(32, 32, 32, "centre", 10.0)
    P = oracle.Problem3(x, y, z)
    f = np.random.default_rng(7).standard_normal(P.shape())
    u = np.zeros(P.shape())
    hist = P.solve(u, f, nu1=2, nu2=2, tol=1e-10, max_cycles=60, smoother="wireframe")
    assert hist[-1] <= 1e-10
    rho_w = (hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1))
    u = np.zeros(P.shape())
    ht = P.solve(u, f, nu1=2, nu2=2, tol=1e-10, max_cycles=60, smoother="tweed")
    rho_t = (ht[-1] / ht[0]) ** (1.0 / (len(ht) - 1))
    assert rho_w < 0.6 and rho_w < 0.8 * rho_t, (rho_w, rho_t)


def test_alternating_is_tweed_then_wireframe_and_converges_on_both_clusterings():
    """Sec. 3's alternating scheme in 3D: one step is a tweed relaxation then
    a wireframe relaxation, and its cycles converge on grids clustered toward
    the walls and toward the centre."""
    P = oracle.Problem3(*grid3(12, 10, 8, "wall", 30.0))
    rng = np.random.default_rng(8)
    u0, f = rng.standard_normal(P.shape()), rng.standard_normal(P.shape())
    a = P.smooth(u0.copy(), f, smoother="alt_tw")
    b = P.smooth(P.smooth(u0.copy(), f, smoother="tweed"), f, smoother="wireframe")
    assert np.array_equal(a, b)
    for kind, ratio in (("wall", 100.0), ("centre", 10.0)):
        P = oracle.Problem3(*grid3(32, 32, 32, kind, ratio))
        u = np.zeros(P.shape())
        h = P.solve(u, f=rng.standard_normal(P.shape()), nu1=2, nu2=2, tol=1e-10, max_cycles=40, smoother="alt_tw")
        assert h[-1] <= 1e-10 and (h[-1] / h[0]) ** (1.0 / (len(h) - 1)) < 0.6, (kind, len(h))


@pytest.mark.parametrize("dims", [(10, 10, 10), (12, 8, 6), (16, 12, 10)])
def test_three_motifs_cover_every_wire_once(dims):
    """Sec. 7: tweed, wireframe and complementary wireframe together hold every
    wire of the grid between interior nodes, each in exactly one motif."""
    P = oracle.Problem3(*grid3(*dims))
    owners = [P.partition(smoother=sm)[0] for sm in ("tweed", "wireframe", "complementary")]
    for k, j, i in interior_nodes(owners[0].shape):
        for di, dj, dk in DIRS[1::2]:
            kk, jj, ii = k + dk, j + dj, i + di
            if owners[0][kk, jj, ii] < 0:
                continue
            held = [int(o[k, j, i] == o[kk, jj, ii]) for o in owners]
            assert sum(held) == 1, ((k, j, i), (kk, jj, ii), held)


@pytest.mark.parametrize("n", [10, 12])
def test_complementary_cube_blocks(n):
    """Sec. 7, complementary wireframe on a cube: the 8 corner points are point
    relaxations (red), and on every concentric cuboid the lines join into one
    block of six "+" shapes centred on the faces (six nodes with four in-block
    neighbours, at the face centres); every other block is a point or a ring."""
    P = oracle.Problem3(*grid3(n, n, n))
    owner, colour = P.partition(smoother="complementary")
    sizes, edges, deg = block_graph(owner)
    for i in (1, n - 1):
        for j in (1, n - 1):
            for k in (1, n - 1):
                b = owner[k, j, i]
                assert sizes[b] == 1 and colour[b] == 0
    c = n // 2
    plus = 0
    for b in range(len(colour)):
        d = deg[owner == b]
        if (d == 4).any():
            plus += 1
            centres = sorted(tuple(p) for p in np.argwhere((owner == b) & (deg == 4)))
            t = min(centres[0])
            expect = sorted([(c, c, t), (c, c, n - t), (c, t, c), (c, n - t, c), (t, c, c), (n - t, c, c)])
            assert centres == expect, (b, centres)
            assert (d[d != 4] == 2).all() and edges[b] == sizes[b] + 6
        else:
            assert sizes[b] == 1 or (edges[b] == sizes[b] and (d == 2).all()), b
    assert plus == sum(1 for t in range(1, c) if n - 2 * t >= 2)


def test_triplet_beats_single_motifs_on_mixed_clustering():
    """Sec. 7: for stretching in several directions the paper proposes
    triplets of sweeps (tweed, wireframe, complementary).  On a grid clustered
    toward the walls in x and toward the centre in y the triplet's V(1,1)
    cycles converge faster than those of any one motif or of the tweed /
    wireframe pair."""
    n = 32
    P = oracle.Problem3(I.coords(n, "wall", ratio=100.0), I.coords(n, "centre", ratio=10.0), I.uniform_coords(n))
    f = np.random.default_rng(9).standard_normal(P.shape())
    rate = {}
    for sm in ("tweed", "wireframe", "complementary", "alt_tw", "triplet"):
        h = P.solve(np.zeros(P.shape()), f, nu1=1, nu2=1, tol=1e-10, max_cycles=12, smoother=sm)
        rate[sm] = (h[-1] / h[0]) ** (1.0 / (len(h) - 1))
    assert rate["triplet"] < 0.9 * min(v for k, v in rate.items() if k != "triplet"), rate
