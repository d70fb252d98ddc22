"""The C-ABI library loads and exports every entry point the header
declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2507_01152_gb300 import build, ussim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^US_API\s+[\w\s\*]+?\b(us_\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    assert "us_sim_create" in names and "us_sim_render" in names and len(names) == len(set(names))


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) == set(ussim.SIGNATURES)


def test_status_strings(lib):
    lib.us_status_string.restype = ctypes.c_char_p
    assert lib.us_status_string(0) == b"US_OK"
    assert lib.us_status_string(1) == b"US_ERR_INVALID_ARG"


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    """Host-side validation: NULL/zero-size arguments fail with
    US_ERR_INVALID_ARG and never reach CUDA."""
    L = ussim.load()
    h = ctypes.c_void_p()
    assert L.us_sim_create(None, 0, None, 0, None, 0, None, ctypes.byref(h)) == ussim.US_ERR_INVALID_ARG
    assert not h.value
    vol = ussim.us_volume(None, None, 4, 4, 4, 1.0)
    tab = (ussim.us_tissue * 1)(ussim.us_tissue(0.5, 1.5, 0.5, 0.1, 0.0))
    pr = (ussim.us_probe * 1)(ussim.us_probe(0, 8, 16, 10.0, 0.5, 0, 0, 8, 16, 5, 1, 0.3, 1, 60))
    assert L.us_sim_create(ctypes.byref(vol), 1, tab, 1, pr, 1, None, ctypes.byref(h)) == ussim.US_ERR_INVALID_ARG


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ussim, "_lib", None)
    with pytest.raises(RuntimeError):
        ussim.load()


def test_env_array_layout():
    """the binding's us_env array is the int32 [B][2] rows, in order (it is
    built by one buffer copy)"""
    import ctypes as C
    import numpy as np
    from paper_2507_01152_gb300.ussim import make_envs, us_env
    assert C.sizeof(us_env) == 8
    e = np.array([[1, 2], [3, 4], [0, 7], [5, 0]], np.int64)        # any integer dtype
    a = make_envs(e)
    assert [(x.volume_id, x.probe_id) for x in a] == [(1, 2), (3, 4), (0, 7), (5, 0)]
    assert [(x.volume_id, x.probe_id) for x in make_envs(e[:, ::-1][:, ::-1])] == [(1, 2), (3, 4), (0, 7), (5, 0)]
    assert len(make_envs(np.zeros((0, 2), np.int32))) == 1          # a valid pointer for an empty batch
