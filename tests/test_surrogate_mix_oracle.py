"""Pins of the oracle's pieces of the surrogate's mixed-probe step (no
GPU): the common-grid slice sampler, the resize back to a probe's own grid,
and the seeded selection of the gate's physics audit."""
import math

import numpy as np

import oracle
from paper_2507_01152_gb300 import scene


def _pose(t):
    return np.array([[1, 0, 0, t[0]], [0, 1, 0, t[1]], [0, 0, 1, t[2]]], np.float32)


def test_grid_slice_at_the_output_size_is_the_output_slice():
    """on a curvilinear probe's own output size the common grid is the
    scan-conversion grid: the same slice as the per-probe sampler"""
    spec = scene.VolumeSpec(64, 64, 64, 1.0, 1, 1000)
    lab, hu = scene.make_volume(spec)
    pr = scene.curvilinear_probe(32, 64, 40.0, 60.0, 20.0, 40, 32)
    pose = scene.dorsal_poses(spec, 1, 3, half_width_mm=10.0, k_margin_mm=10.0)[0]
    a = oracle.sample_slice(lab, hu, spec.voxel_mm, pr, pose)
    b = oracle.sample_slice_grid(lab, hu, spec.voxel_mm, pr, pose, pr.out_h, pr.out_w)
    np.testing.assert_array_equal(a, b)


def test_grid_slice_linear_axis_aligned_closed_form():
    """linear probe, identity rotation, a volume whose label is the voxel's
    k index mod 5 and whose HU is 100 k: the grid pixel (r, c) sits at
    depth ((r + 1/2) NS / H - 1/2) dr below t, so its nearest k and its
    trilinear HU follow by hand (dyadic values: exact in FP32)"""
    nz, ny, nx = 64, 8, 8
    k = np.arange(nz)
    lab = np.broadcast_to((k % 5).astype(np.uint8)[:, None, None], (nz, ny, nx)).copy()
    hu = np.broadcast_to((100 * k).astype(np.int16)[:, None, None], (nz, ny, nx)).copy()
    pr = scene.linear_probe(4, 64, 32.0, 0.5)           # dr = 0.5 mm
    t = (4.0, 4.0, 2.0)
    out = oracle.sample_slice_grid(lab, hu, 1.0, pr, _pose(t), 32, 8)
    for r in range(32):
        z = ((r + 0.5) * 64 / 32 - 0.5) * 0.5 + t[2]    # mm = voxel units (h = 1 mm)
        kk = math.floor(z + 0.5)
        assert np.all(out[r, :, 0] == (kk % 5) / 4.0)
        assert np.allclose(out[r, :, 1], min(max(100 * z / 1000.0, -1), 3), rtol=0, atol=1e-12)
        assert np.all(out[r, :, 2] == 1.0)
    # lateral positions: ((c + 1/2) NL / W - 1/2 - (NL - 1) / 2) pitch
    xs = [((c + 0.5) * 4 / 8 - 0.5 - 1.5) * 0.5 for c in range(8)]
    assert xs[0] == -0.875 and xs[-1] == 0.875


def test_resize_reproduces_linear_functions_and_is_identity_at_the_same_size():
    pr = scene.linear_probe(96, 160, 80.0, 0.5)         # output 160 x 96
    H, W = 64, 48
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    src = 2.0 * yy + 3.0 * xx
    out = oracle.resize_frame(src, pr)
    for r in (0, 1, 37, 159):
        fy = min(max((r + 0.5) * H / 160 - 0.5, 0), H - 1)
        for c in (0, 5, 95):
            fx = min(max((c + 0.5) * W / 96 - 0.5, 0), W - 1)
            assert abs(out[r, c] - (2 * fy + 3 * fx)) < 1e-12
    same = np.random.default_rng(1).random((160, 96))
    np.testing.assert_allclose(oracle.resize_frame(same, pr), same, rtol=0, atol=1e-15)


def test_resize_zeroes_outside_the_fan():
    pr = scene.curvilinear_probe(64, 128, 60.0, 60.0, 30.0, 48, 40)
    m = oracle.fan_mask(pr)
    assert 0.3 < m.mean() < 0.95
    out = oracle.resize_frame(np.ones((32, 32)), pr, m)
    assert np.all(out[~m] == 0) and np.allclose(out[m], 1.0)


def test_audit_selection_rate_and_exclusion():
    """the audit takes about the stated fraction of the frames the gate
    keeps, none of the gated ones, all of the kept ones at fraction 1 and
    none at 0; the selection changes with the step"""
    B = 20000
    rng = np.random.default_rng(4)
    score = rng.random(B)
    thr = 0.9
    sel = oracle.audit_selected(B, 77, 3, 0.05, score, thr)
    kept = ~(score > thr)
    assert not np.any(sel & ~kept)
    n = kept.sum()
    assert abs(sel.sum() / n - 0.05) < 5 * math.sqrt(0.05 * 0.95 / n)
    assert np.array_equal(oracle.audit_selected(200, 77, 3, 1.0, score[:200], thr), kept[:200])
    assert not oracle.audit_selected(200, 77, 3, 0.0, score[:200], thr).any()
    other = oracle.audit_selected(B, 77, 4, 0.05, score, thr)
    assert (other != sel).sum() > 0.05 * n
