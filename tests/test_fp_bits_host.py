"""The integer-pipe conversions of the refinement kernels (csrc/fp_bits.h),
on the CPU.  narrow_rne (binary64 -> binary32, round to nearest, ties to
even) must give the compiler's own conversion bit for bit on ties either
way, carries into the exponent and out of the subnormal range, the largest
finite float, subnormal results and the rounding to zero below them, zeros,
Inf, NaN and four million random doubles over every exponent the float range
reaches and beyond; widen_exact (binary32 -> binary64) on all 2^32 floats.
A dropped tie rule (round half up), a lost carry or a subnormal
normalised off by one fails it."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_conversions_match_the_compilers(tmp_path):
    exe = tmp_path / "fp_bits_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(ROOT, "tests", "fp_bits_driver.cpp"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe), "4000000"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > (1 << 32) + 4000000
