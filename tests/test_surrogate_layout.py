"""The library's surrogate parameter layout equals the oracle's (host-only
queries, no GPU)."""
import math

import numpy as np

from oracle import surrogate_ref as S
from paper_2507_01152_gb300 import scene
from paper_2507_01152_gb300.ussim import Surrogate


def test_parameter_segments_match_oracle():
    for c in (16, 32):
        off, size, fan = Surrogate.segments(c)
        shapes = S.param_shapes(c)
        assert len(shapes) == len(off)
        o = 0
        for (name, shp), a, n, f in zip(shapes, off, size, fan):
            assert a == o and n == math.prod(shp), name
            if name.endswith(".b"):
                assert f == 0
            else:
                assert f == (shp[1] * shp[2] * shp[3] if len(shp) == 4 else shp[-1]), name
            o += n
        assert Surrogate.num_params(c) == S.n_params(c) == o


def test_init_is_seeded():
    off, size, fan = Surrogate.segments(16)
    a = scene.surrogate_init(size, fan, 3)
    b = scene.surrogate_init(size, fan, 3)
    assert np.array_equal(a, b) and a.size == S.n_params(16)
    assert np.all(a[off[1]:off[1] + size[1]] == 0)
