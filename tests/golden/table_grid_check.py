"""Evidence for the grid-size reading of Tables 1-4 (Sec. 5): the oracle's
two-grid spectral radii on the grids of nx = ny = 64 and 128 intervals, for
all 288 printed entries (tests/golden/twogrid_tables.txt), written to
tests/golden/twogrid_tables_nx64_nx128.txt with, per table, the largest
difference from the printed value in units of the fourth digit.  Calls only
the oracle.

    python tests/golden/table_grid_check.py [processes]
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "twogrid_tables_nx64_nx128.txt")


def rows():
    out = []
    for line in open(os.path.join(HERE, "twogrid_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, g, rs, sm, *vals = line.split()
        out.append((int(t), g, rs, sm, [float(v) for v in vals]))
    return out


def entry(args):
    n, g, rs, sm, nu = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2110_08389_gb300 import inputs as I
    oracle.threads(1)  # one process per core already
    grid = {"uniform": lambda: I.uniform_coords(n), "wall1.5": lambda: I.wall_coords(n, 1.5),
            "wall3.0": lambda: I.wall_coords(n, 3.0), "centre1.5": lambda: I.centre_coords(n, 1.5)}[g]()
    P = oracle.Problem(grid, grid)
    smo = "zebra_x" if sm == "zebra" else sm
    return P.twogrid_radius(smo, oracle.HW if rs == "HW" else oracle.FW, nu, 0)


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    rs = rows()
    jobs = [(n, g, r, sm, nu) for n in (64, 128) for (t, g, r, sm, _) in rs for nu in range(1, 7)]
    with mp.get_context("spawn").Pool(procs) as pool:
        vals = pool.map(entry, jobs, chunksize=1)
    got = dict(zip(jobs, vals))
    lines = ["# Two-grid spectral radius rho(M) of the oracle (Eq. Mh2h) on the grids of nx = ny = 64 and 128",
             "# intervals, against the values printed in Tables 1-4 (tests/golden/twogrid_tables.txt).",
             "# Written by tests/golden/table_grid_check.py.",
             "# Columns: table grid restriction smoother nu printed rho(nx=64) rho(nx=128)"]
    worst = {}
    for (t, g, r, sm, printed) in rs:
        for nu in range(1, 7):
            a, b = got[(64, g, r, sm, nu)], got[(128, g, r, sm, nu)]
            p = printed[nu - 1]
            lines.append(f"{t} {g} {r} {sm} {nu} {p:.4f} {a:.6f} {b:.6f}")
            for n, v in ((64, a), (128, b)):
                d = abs(round(v, 4) - p) * 1e4
                key = (t, n)
                cnt, mx = worst.get(key, (0, 0.0))
                worst[key] = (cnt + (d > 0.5), max(mx, d))
    lines.append("# per table: entries (of 72) whose four-digit rounding differs from the printed value, and the")
    lines.append("# largest difference in units of the fourth digit")
    for t in (1, 2, 3, 4):
        for n in (64, 128):
            cnt, mx = worst[(t, n)]
            lines.append(f"# table {t} nx={n}: {cnt} differ, max {mx:.0f}")
    open(OUT, "w").write("\n".join(lines) + "\n")
    print("\n".join(lines[-9:]))


if __name__ == "__main__":
    main()
