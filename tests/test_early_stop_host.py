"""The early-stop rule of mg_params.early_stop (csrc/solve.h), on the CPU:
never before the third step or without a previous step, always when a step
did not reduce the residual, and otherwise exactly when the last step's
rate, kept for the steps the caps leave, cannot reach the tolerance; and the
count of steps the caps leave (expected values worked by hand)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # steps, rel, prev, left, tol, give up?
    (2, 1e-2, 1e-3, 10, 1e-10, 0),   # too early, although the residual grew
    (3, 1e-3, 1e-3, 10, 1e-10, 1),   # no reduction
    (3, 2e-3, 1e-3, 10, 1e-10, 1),   # growth
    (3, 1e-3, 1e-2, 6, 1e-10, 1),    # rate 0.1 for 6 steps: 1e-9 > 1e-10
    (3, 1e-3, 1e-2, 8, 1e-10, 0),    # rate 0.1 for 8 steps: 1e-11
    (5, 0.5, 0.6, 100, 1e-10, 1),    # (5/6)^100 * 0.5 = 6e-9
    (5, 0.5, 0.6, 150, 1e-10, 0),    # (5/6)^150 * 0.5 = 7e-13
    (4, 1e-4, 0.0, 1, 1e-10, 0),     # no previous step
]


# Steps left under the caps.  An FP32+refine step runs all inner_cycles and
# the caps are checked after it, so a step still starts while cycles <
# max_cycles: with max_cycles = 100 and 3 inner cycles, 96 cycles leave two
# steps (96 -> 99 -> 102), not one.
LEFT = [  # f64, max_cycles, max_outer, inner, cycles, outer, steps left
    (1, 100, 8, 3, 96, 0, 4),
    (1, 100, 8, 3, 100, 0, 0),
    (0, 100, 50, 3, 96, 32, 2),     # max_cycles not a multiple of inner_cycles
    (0, 100, 50, 3, 99, 33, 1),
    (0, 100, 50, 3, 102, 34, 0),
    (0, 99, 50, 3, 96, 32, 1),      # a multiple: exactly one more step
    (0, 100, 33, 3, 96, 32, 1),     # the outer cap binds
    (0, 100, 8, 4, 0, 0, 8),
    (0, 10, 8, 4, 0, 0, 3),         # 0 -> 4 -> 8 -> 12
]


def _driver(tmp_path):
    exe = tmp_path / "early_stop_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", "/usr/local/cuda/include", os.path.join(ROOT, "tests", "early_stop_driver.cpp"),
                    "-o", str(exe)], check=True)
    return exe


def test_hopeless_rule(tmp_path):
    exe = _driver(tmp_path)
    inp = "\n".join(f"h {s} {r!r} {p!r} {l} {t!r}" for s, r, p, l, t, _ in CASES) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [c[-1] for c in CASES]


def test_steps_left(tmp_path):
    exe = _driver(tmp_path)
    inp = "\n".join("s " + " ".join(str(v) for v in c[:-1]) for c in LEFT) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [c[-1] for c in LEFT]


def test_steps_left_matches_a_simulated_solve(tmp_path):
    """steps_left equals the steps a solve that never converges goes on to
    run, counted by simulating the caps: a step starts while cycles <
    max_cycles and outer < max_outer, and adds inner_cycles and one step."""
    import itertools
    exe = _driver(tmp_path)
    cases, want = [], []
    for mc, mo, inner in itertools.product((7, 9, 10, 12), (2, 3, 5), (1, 2, 3, 4)):
        cycles = outer = 0
        while True:
            c, o, n = cycles, outer, 0
            while c < mc and o < mo:
                c += inner
                o += 1
                n += 1
            cases.append(f"s 0 {mc} {mo} {inner} {cycles} {outer}")
            want.append(n)
            if n == 0:
                break
            cycles += inner
            outer += 1
    out = subprocess.run([str(exe)], input="\n".join(cases) + "\n", capture_output=True, text=True,
                         check=True).stdout.split()
    assert [int(v) for v in out] == want
