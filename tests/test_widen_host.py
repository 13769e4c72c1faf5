"""The refinement update widens the FP32 correction to FP64 from its IEEE-754
fields (csrc/transfer.cu, widen): sign, exponent rebiased by 1023 - 127 = 896,
mantissa moved up 29 bits, with zero, subnormal and non-finite floats left to
the conversion instruction.  The same bit formula, applied here to normal
floats of every exponent and both signs, must give exactly numpy's widening."""
import numpy as np


def widen_fields(x):
    b = x.view(np.uint32).astype(np.uint64)
    ex = (b >> np.uint64(23)) & np.uint64(0xFF)
    bits = ((b & np.uint64(0x80000000)) << np.uint64(32)) | ((ex + np.uint64(896)) << np.uint64(52)) | \
           ((b & np.uint64(0x7FFFFF)) << np.uint64(29))
    return bits.view(np.float64)


def test_widen_fields_match_numpy():
    rng = np.random.default_rng(5)
    ex = rng.integers(1, 255, size=200000).astype(np.uint32)  # every normal exponent
    mant = rng.integers(0, 1 << 23, size=200000).astype(np.uint32)
    sign = rng.integers(0, 2, size=200000).astype(np.uint32)
    x = ((sign << 31) | (ex << 23) | mant).view(np.float32)
    edges = np.array([np.finfo(np.float32).tiny, -np.finfo(np.float32).tiny, np.finfo(np.float32).max,
                      -np.finfo(np.float32).max, 1.0, -1.0, 1.5e-30, 3.0e30], dtype=np.float32)
    x = np.concatenate([x, edges])
    assert np.array_equal(widen_fields(x), x.astype(np.float64))
