"""Integer results the render kernels take from FP32 arithmetic.

Pass A spreads the labels of a group's halo lines over its warps as units
t = c * nh + h (c: 32-sample chunk, h: halo line, nh <= 16 halo lines, at
most 32 chunks), and recovers c = t / nh as floor((t + 1/2) * fl(1/nh)) in
FP32: (t + 1/2) / nh lies at least 1 / (2 nh) from an integer, far beyond
the rounding error of one product (or of one fused multiply-add, if the
compiler contracts the sum into it).  Checked here for every t and nh the
kernel can meet, in both forms, with IEEE single arithmetic."""
import numpy as np


def test_halo_unit_quotient_is_exact():
    for nh in range(1, 17):
        inv = np.float32(1.0) / np.float32(nh)
        t = np.arange(nh * 32, dtype=np.int64)
        tf = t.astype(np.float32)
        # separate add and multiply, each rounded to FP32
        c_mul = np.floor((tf + np.float32(0.5)) * inv).astype(np.int64)
        # one fused multiply-add: t * inv + 0.5 * inv rounded once
        fused = (t.astype(np.float64) * np.float64(inv) + np.float64(np.float32(0.5) * inv)).astype(np.float32)
        c_fma = np.floor(fused).astype(np.int64)
        assert np.array_equal(c_mul, t // nh), nh
        assert np.array_equal(c_fma, t // nh), nh
