"""The checked build (build.py --checked, -DMG_CHECK): its kernels validate
every index they decode from their descriptors and record a bad one instead
of using it.  The small-grid parity set runs once on that build in a child
process (tests/checked_run.py): colour passes of every smoother and path
with the relaxed colour's own nodes set to NaN beforehand (a pass must not
read them), transfers into NaN-filled outputs, FP64 and FP32+refine solves,
3D solves and a batch.  Every call must return MG_OK and match the oracle,
and no kernel may have recorded a bad index.  This stands in for a memory
checker where none can be run."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_the_parity_set_clean(mg):
    from paper_2110_08389_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, TWEEDMG_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    last = [ln for ln in r.stderr.splitlines() if ln.strip()][-3:] if r.stderr else []
    assert r.returncode == 0, (r.stdout[-1000:], last)
    assert "checked ok" in r.stdout
