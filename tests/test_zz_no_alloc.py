"""us_sim_render_plain_static: the render entry point that allocates
nothing, for callers that must not allocate device memory while they
render.  Its scratch is a fixed array compiled into the library, so its
frames must equal those of us_sim_render_plain (same kernels) call after
call, even though every call reuses the same scratch."""
import numpy as np
import pytest

from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sim_and_inputs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    from paper_2507_01152_gb300.ussim import Sim
    build.build()
    spec = scene.VolumeSpec(128, 128, 128, 0.75, 2, 1000)
    lab, hu = scene.make_volume(spec)
    # the curvilinear probe is exactly at the static scratch limit (256 x 512 samples)
    probes = [scene.curvilinear_probe(256, 512, 60.0, 60.0, 30.0, 192, 160),
              scene.linear_probe(96, 200, 50.0, 0.5),
              scene.curvilinear_probe(512, 512, 60.0, 60.0, 30.0, 64, 64)]   # over the limit
    sim = Sim([(torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), spec.voxel_mm)], scene.tissue_table(),
              probes, scene.Options())
    return sim, spec


def _render(fn, sim, envs, poses, seed, step):
    off = sim.frame_layout(envs)
    frames = torch.full((int(off[-1]),), -5.0, dtype=torch.float32, device="cuda")
    fn(envs, poses, seed, step, frames)
    torch.cuda.synchronize()
    return frames.cpu().numpy()


def test_static_scratch_matches_allocating_path_two_calls(sim_and_inputs):
    sim, spec = sim_and_inputs
    B = 6
    envs = np.array([[0, b % 2] for b in range(B)], np.int32)
    poses_a = torch.from_numpy(scene.dorsal_poses(spec, B, 31, half_width_mm=20.0, k_margin_mm=20.0)).cuda()
    poses_b = torch.from_numpy(scene.dorsal_poses(spec, B, 32, half_width_mm=20.0, k_margin_mm=20.0)).cuda()
    ref_a = _render(sim.render_plain, sim, envs, poses_a, 77, 1)
    ref_b = _render(sim.render_plain, sim, envs[::-1].copy(), poses_b, 78, 2)
    got_a = _render(sim.render_plain_static, sim, envs, poses_a, 77, 1)
    free_before, _ = torch.cuda.mem_get_info()
    got_b = _render(sim.render_plain_static, sim, envs[::-1].copy(), poses_b, 78, 2)
    free_after, _ = torch.cuda.mem_get_info()
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        assert np.abs(got - ref).max() <= 1e-3          # the frame tolerance of the parity tests
        assert np.array_equal(got, ref)                 # same kernels: identical in fact
    assert np.any(got_a > 0) and np.any(got_b > 0)
    assert free_after == free_before                    # the second call allocated no device memory


def test_static_scratch_rejects_beam_grids_over_the_limit(sim_and_inputs):
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_INVALID_ARG
    sim, spec = sim_and_inputs
    envs = np.array([[0, 2]], np.int32)
    poses = torch.from_numpy(scene.dorsal_poses(spec, 1, 33, half_width_mm=20.0, k_margin_mm=20.0)).cuda()
    frames = torch.zeros(64 * 64, device="cuda")
    with pytest.raises(UsError) as e:
        sim.render_plain_static(envs, poses, 1, 1, frames)
    assert e.value.status == US_ERR_INVALID_ARG
    assert "131072" in str(e.value)
