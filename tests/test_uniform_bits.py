"""The kernels' uniform variate: for the top 23 bits k of a Philox word they
form (2k + 1) 2^-24 as (1 + k 2^-23) - (1 - 2^-24), the float with exponent
0 and mantissa k less a constant.  The difference is representable, so the
FP32 subtraction is exact: checked here for every k with IEEE single
arithmetic (numpy float32), against the odd multiple of 2^-24 formed
directly in FP64."""
import numpy as np


def test_uniform_from_mantissa_bits_is_exact_for_every_k():
    k = np.arange(1 << 23, dtype=np.uint32)
    one_plus = (np.uint32(0x3F800000) | k).view(np.float32)
    got = one_plus - np.float32(1.0 - 2.0 ** -24)
    assert got.dtype == np.float32
    want = (2.0 * k.astype(np.float64) + 1.0) * 2.0 ** -24
    assert np.array_equal(got.astype(np.float64), want)
    assert got.min() > 0 and got.max() < 1
