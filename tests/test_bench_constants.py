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
