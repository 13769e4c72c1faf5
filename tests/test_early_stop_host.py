"""The early-stop rule of mg_params.early_stop (csrc/solve.h), on the CPU:
never before the third step or without a previous step, always when a step
did not reduce the residual, and otherwise exactly when the last step's
rate, kept for the steps the caps leave, cannot reach the tolerance
(expected values worked by hand)."""
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


def test_hopeless_rule(tmp_path):
    exe = tmp_path / "early_stop_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2110_08389_gb300", "csrc"),
                    "-I", "/usr/local/cuda/include", os.path.join(ROOT, "tests", "early_stop_driver.cpp"),
                    "-o", str(exe)], check=True)
    inp = "\n".join(f"{s} {r!r} {p!r} {l} {t!r}" for s, r, p, l, t, _ in CASES) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [c[-1] for c in CASES]
