"""Reconstruction observation of the bone-surface task (Task 2 with App. C):
the oracle pinned to closed forms - the missing-point rate, the surface of a
planar bone slab, and the voxelization of single points under known poses."""
import math

import numpy as np

import oracle
from paper_2507_01152_gb300 import scene

BONE = 4


def _slab(k0, shape=(60, 24, 40)):
    lab = np.full(shape, 3, np.uint8)      # muscle
    lab[k0:] = BONE                        # bone for z index >= k0
    return lab, np.zeros(shape, np.int16)


def _pose(R, t):
    return np.concatenate([np.asarray(R, np.float32), np.asarray(t, np.float32)[:, None]], axis=1)


def test_planar_bone_surface_points_sit_on_the_slab_face():
    """Probe looking along +z at a bone slab from z index 30: each line meets
    the surface once, at voxel z = 30; with no misses every point is kept."""
    lab, hu = _slab(30)
    pr = scene.linear_probe(16, 160, 40.0, 0.5)             # lines along x, 0.25 mm samples
    P = _pose(np.eye(3), (8.0, 5.0, 2.0))
    rec = np.zeros_like(lab)
    n, kept = oracle.recon_update(lab, hu, 0.5, pr, P, 0, 1, 0, BONE, 0.0, rec)
    assert n == 16 and kept == 16
    z, y, x = np.nonzero(rec)
    assert np.all(z == 30) and np.all(y == 10) and len(np.unique(x)) == len(x)


def test_missing_points_follow_the_miss_probability():
    lab, hu = _slab(30, (60, 24, 160))
    pr = scene.linear_probe(150, 160, 40.0, 0.5)
    total = kept = 0
    for step in range(40):
        rec = np.zeros_like(lab)
        n, k = oracle.recon_update(lab, hu, 0.5, pr, _pose(np.eye(3), (40.0, 5.0, 2.0)), 3, 9, step, BONE, 0.2, rec)
        total += n
        kept += k
    frac = kept / total
    assert abs(frac - 0.8) < 5 * math.sqrt(0.16 / total), (frac, total)
    assert oracle.recon_keep_threshold(0.2) == int(0.2 * 2 ** 32)


def test_observation_voxelizes_points_in_the_probe_frame():
    """One reconstructed voxel at (ix, jy, kz) (0.5 mm voxels): identity pose
    puts it at (h, w, e) = (floor(z / 3), floor(x / 3) + 20, floor(y / 3) + 20);
    the probe moved 3 mm along its x shifts it one column; a quarter turn
    about z swaps the lateral and elevation axes."""
    rec = np.zeros((60, 30, 40), np.uint8)
    ix, jy, kz = 13, 7, 50                                  # x = 6.5, y = 3.5, z = 25 mm
    rec[kz, jy, ix] = 1
    o = oracle.recon_observe(rec, 0.5, _pose(np.eye(3), (0, 0, 0)))
    assert list(zip(*np.nonzero(o))) == [(8, 22, 21)]
    o = oracle.recon_observe(rec, 0.5, _pose(np.eye(3), (3.0, 0, 0)))
    assert list(zip(*np.nonzero(o))) == [(8, 21, 21)]
    R = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]                  # probe x -> volume y, probe y -> volume -x
    o = oracle.recon_observe(rec, 0.5, _pose(R, (0, 0, 0)))
    # q = R^T p = (y, -x, z) = (3.5, -6.5, 25)
    assert list(zip(*np.nonzero(o))) == [(8, 21, 17)]
    assert oracle.recon_observe(rec, 0.5, _pose(np.eye(3), (0, 0, 200.0))).sum() == 0   # behind the probe
