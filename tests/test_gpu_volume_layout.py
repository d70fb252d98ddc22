"""Corner records of the HU grid (the 8 corners of a trilinear cell in one
16-byte record): images identical to those read from the caller's grid on
every path, including samples whose cells straddle the grid's faces, and
us_sim_refresh_volumes after the caller changes a volume."""
import dataclasses

import numpy as np
import pytest

from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()


def _sim(wl, lab, hu, layout, options=None):
    from paper_2507_01152_gb300.ussim import Sim
    opt = dataclasses.replace(options or wl.options, volume_layout=layout)
    return Sim([(lab, hu, wl.volumes[0][0].voxel_mm)], scene.tissue_table(), wl.probes, opt)


def _render(sim, envs, poses, step, shape=None, plain=False):
    from simhelp import render_gpu
    if shape is not None:
        sim.set_tuning(shape[0], shape[1], 0)
    return render_gpu(sim, envs, poses, 11, step, path=1 if plain else 0)


def _edge_poses(spec, n):
    """Poses whose images run past the grid's faces: the dorsal poses shifted
    sideways and along the spine by up to half the volume."""
    poses = scene.dorsal_poses(spec, n, 77).copy()
    ext = np.array([spec.nx, spec.ny, spec.nz], np.float32) * spec.voxel_mm
    for b in range(n):
        poses[b, :, 3] += (b % 3 - 1) * 0.45 * ext
    return poses


@pytest.mark.parametrize("opt", [scene.Options(), scene.Options(z_mode=0, speckle=0, transmission=1)])
def test_layouts_give_identical_images(opt):
    wl = scene.workload_c2(6)
    spec, lab_np, hu_np = wl.volumes[0]
    lab, hu = torch.from_numpy(lab_np).cuda(), torch.from_numpy(hu_np).cuda()
    envs = wl.envs[:6]
    poses = _edge_poses(spec, 6)
    a, b = _sim(wl, lab, hu, 0, opt), _sim(wl, lab, hu, 1, opt)
    for kw in (dict(shape=(1, 16)), dict(shape=(8, 32)), dict(plain=True)):
        ga, gb = _render(a, envs, poses, 3, **kw), _render(b, envs, poses, 3, **kw)
        for e in range(6):
            for k in ("frame", "envelope", "logimg", "nn_index", "label"):
                assert np.array_equal(ga[e][k], gb[e][k]), (kw, e, k)
    # the shifted poses really reach past the grid (label 0 outside)
    assert any((g["nn_index"] < 0).mean() > 0.05 for g in ga)
    a.close()
    b.close()


def test_refresh_volumes_after_the_hu_grid_changes():
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_INVALID_ARG
    wl = scene.workload_c2(4)
    spec, lab_np, hu_np = wl.volumes[0]
    lab, hu = torch.from_numpy(lab_np).cuda(), torch.from_numpy(hu_np).cuda()
    envs, poses = wl.envs[:4], wl.poses[:4]
    sim = _sim(wl, lab, hu, 0)
    before = _render(sim, envs, poses, 2, shape=(1, 16))
    hu[:, :, : spec.nx // 2] += 200          # a brighter half volume
    sim.refresh_volumes()
    after = _render(sim, envs, poses, 2, shape=(1, 16))
    fresh = _sim(wl, lab, hu, 1)
    want = _render(fresh, envs, poses, 2, shape=(1, 16))
    for e in range(4):
        assert np.array_equal(after[e]["envelope"], want[e]["envelope"])
        assert np.array_equal(after[e]["frame"], want[e]["frame"])
    assert any(not np.array_equal(before[e]["envelope"], after[e]["envelope"]) for e in range(4))
    # a label outside the tissue table is refused at refresh
    keep = int(lab[0, 0, 0])
    lab[0, 0, 0] = 250
    with pytest.raises(UsError) as ei:
        sim.refresh_volumes()
    assert ei.value.status == US_ERR_INVALID_ARG
    lab[0, 0, 0] = keep
    sim.refresh_volumes()
    sim.close()
    fresh.close()


def test_bricked_labels_and_corner_quads_on_a_ragged_grid():
    """A grid whose sides are not multiples of 4 (the label bricks and the
    corner records' y quads then end in padding): every render path, the
    surrogate's slice sampling on the beam grid and on a square grid, and
    the exported labels and voxel indices equal those read from the caller's
    grid, with poses that run past every face."""
    spec = scene.VolumeSpec(126, 130, 122, 1.0, 2, 4321)
    lab_np, hu_np = scene.make_volume(spec)
    wl = scene.Workload("ragged", [(spec, lab_np, hu_np)], [scene.curvilinear_probe(96, 192, 80.0, 60.0, 40.0, 96, 96),
                                                           scene.linear_probe(64, 128, 80.0, 0.5)],
                        np.array([[0, b % 2] for b in range(8)], np.int32), _edge_poses(spec, 8), seed=5)
    lab, hu = torch.from_numpy(lab_np).cuda(), torch.from_numpy(hu_np).cuda()
    a, b = _sim(wl, lab, hu, 0), _sim(wl, lab, hu, 1)
    for kw in (dict(shape=(1, 16)), dict(shape=(1, 8)), dict(shape=(8, 32)), dict(plain=True)):
        ga, gb = _render(a, wl.envs, wl.poses, 4, **kw), _render(b, wl.envs, wl.poses, 4, **kw)
        for e in range(8):
            for k in ("frame", "envelope", "logimg", "nn_index", "label"):
                assert np.array_equal(ga[e][k], gb[e][k]), (kw, e, k)
    assert any((g["nn_index"] < 0).mean() > 0.05 for g in ga)
    P = torch.from_numpy(np.ascontiguousarray(wl.poses, np.float32)).cuda()
    for H, W in ((64, 64), (37, 53)):
        sa = torch.empty((8, H, W, 8), dtype=torch.bfloat16, device="cuda")
        sb = torch.empty_like(sa)
        a.sample_slices_grid(wl.envs, P, H, W, sa)
        b.sample_slices_grid(wl.envs, P, H, W, sb)
        torch.cuda.synchronize()
        assert torch.equal(sa.view(torch.int16), sb.view(torch.int16))
        assert float(sa[..., 0].float().max()) > 0      # labels were read
    a.close()
    b.close()


def test_refresh_volumes_after_the_labels_change():
    """us_sim_refresh_volumes rebuilds the bricked labels: a relabelled block
    renders as a fresh handle reading the caller's grid renders it."""
    wl = scene.workload_c2(4)
    spec, lab_np, hu_np = wl.volumes[0]
    lab, hu = torch.from_numpy(lab_np.copy()).cuda(), torch.from_numpy(hu_np).cuda()
    envs, poses = wl.envs[:4], wl.poses[:4]
    sim = _sim(wl, lab, hu, 0)
    before = _render(sim, envs, poses, 2, shape=(1, 16))
    lab[:, 60:200, 40:90] = 4           # a block of bone
    sim.refresh_volumes()
    after = _render(sim, envs, poses, 2, shape=(1, 16))
    fresh = _sim(wl, lab, hu, 1)
    want = _render(fresh, envs, poses, 2, shape=(1, 16))
    for e in range(4):
        for k in ("label", "envelope", "frame"):
            assert np.array_equal(after[e][k], want[e][k]), (e, k)
    assert any(not np.array_equal(before[e]["label"], after[e]["label"]) for e in range(4))
    sim.close()
    fresh.close()
