"""The benchmark's algorithmic byte count is the oracle's exact count."""
import oracle
from paper_2507_01152_gb300 import scene

import bench


def test_c2_touched_voxels_constant():
    wl = scene.workload_c2(64)
    spec, lab, hu = wl.volumes[0]
    tot, per = oracle.touched_voxels([(lab, hu, spec.voxel_mm)], wl.probes, wl.envs, wl.poses)
    assert tot == bench.C2_TOUCHED_VOXELS_VALUE
    assert bench.c2_launch_bytes(64) == 3 * tot + 64 * 256 * 256 * 4 + 64 * 48


def test_c3_touched_voxels_constant():
    """the 512-env batch over four 512 x 512 x 256 volumes (first step of its
    random walks): about 10 s to build the volumes, 8 s to count"""
    wl = scene.workload_c3(512, steps=1)
    vols = [(lab, hu, spec.voxel_mm) for (spec, lab, hu) in wl.volumes]
    tot, per = oracle.touched_voxels(vols, wl.probes, wl.envs, wl.poses[0])
    assert tot == bench.C3_TOUCHED_VOXELS_VALUE
    wl.poses = wl.poses[0]
    px = sum(wl.probes[p].out_w * wl.probes[p].out_h for p in wl.envs[:, 1])
    assert bench.c3_launch_bytes(wl) == 3 * tot + 4 * px + 512 * 48
