"""The surrogate's mixed-probe step on the GPU against the oracle: slices
on a common grid for every probe type, the resize back to each probe's own
grid, and the gate's seeded physics audit."""
import numpy as np
import pytest

import oracle
from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    from paper_2507_01152_gb300.ussim import Sim
    build.build()
    spec = scene.VolumeSpec(160, 160, 128, 0.75, 3, 1007)
    lab, hu = scene.make_volume(spec)
    probes = [scene.linear_probe(64, 128, 60.0, 0.5),                      # output 128 x 64
              scene.curvilinear_probe(96, 192, 60.0, 60.0, 30.0, 96, 96),
              scene.curvilinear_probe(128, 256, 60.0, 60.0, 30.0, 128, 128)]
    sim = Sim([(torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), spec.voxel_mm)], scene.tissue_table(),
              probes, scene.Options())
    B = 9
    envs = np.array([[0, b % 3] for b in range(B)], np.int32)
    poses = scene.dorsal_poses(spec, B, 61, half_width_mm=20.0, k_margin_mm=20.0)
    yield sim, spec, lab, hu, probes, envs, poses
    sim.close()


def test_grid_slices_match_oracle(mix):
    sim, spec, lab, hu, probes, envs, poses = mix
    H, W = 64, 48
    B = len(envs)
    out = torch.zeros((B, H, W, 8), dtype=torch.bfloat16, device="cuda")
    sim.sample_slices_grid(envs, torch.from_numpy(poses).cuda(), H, W, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for b in range(B):
        ref = oracle.sample_slice_grid(lab, hu, spec.voxel_mm, probes[envs[b][1]], poses[b], H, W)
        assert np.array_equal(got[b, ..., 0], ref[..., 0]), b                 # label / 4 (exact in BF16)
        assert np.array_equal(got[b, ..., 2], ref[..., 2]), b                 # inside-field flag
        assert np.all(np.abs(got[b, ..., 1] - ref[..., 1]) <= 2 ** -8 * np.abs(ref[..., 1]) + 1e-6), b
        assert np.all(got[b, ..., 3:] == 0)
        assert (ref[..., 0] > 0).mean() > 0.2


def test_resize_matches_oracle(mix):
    sim, spec, lab, hu, probes, envs, poses = mix
    B = len(envs)
    H, W = 40, 56
    src = torch.rand((B, H, W), generator=torch.Generator().manual_seed(3)).cuda()
    off = sim.frame_layout(envs)
    frames = torch.full((int(off[-1]),), -1.0, device="cuda")
    sim.resize_frames(envs, src, frames)
    torch.cuda.synchronize()
    f = frames.cpu().numpy()
    s = src.double().cpu().numpy()
    for b in range(B):
        pr = probes[envs[b][1]]
        ref = oracle.resize_frame(s[b], pr)
        got = f[off[b]:off[b] + pr.out_h * pr.out_w].reshape(pr.out_h, pr.out_w)
        # the kernel forms the source coordinate in FP32: a few ulps of a
        # coordinate up to H (2^-23 * 64 = 7.6e-6 per ulp) times the largest
        # neighbour difference of the source (1 for these uniform values)
        assert np.abs(got - ref).max() <= 2e-5, (b, np.abs(got - ref).max())


def test_audit_matches_oracle_and_renders_physics(mix):
    """the audited set equals the oracle's seeded selection, each audited
    frame equals the plain physics render of its env, and the frames
    outside the audit stay untouched"""
    sim, spec, lab, hu, probes, envs, poses = mix
    B = len(envs)
    P = torch.from_numpy(poses).cuda()
    score = torch.tensor([0.01, 0.9, 0.02, 0.03, 0.04, 0.95, 0.0, 0.02, 0.01], device="cuda")
    off = sim.frame_layout(envs)
    ref = torch.zeros(int(off[-1]), device="cuda")
    sim.render_plain(envs, P, 55, 6, ref)
    sc = score.cpu().numpy()
    for fraction in (1.0, 0.5):
        audit = torch.full((int(off[-1]),), -3.0, device="cuda")
        flags = torch.zeros(B, dtype=torch.uint8, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        sim.render_audit(envs, P, 55, 6, audit, score, 0.5, fraction, flags, n)
        sim.check()
        want = oracle.audit_selected(B, 55, 6, fraction, sc, 0.5)
        fl = flags.cpu().numpy().astype(bool)
        assert np.array_equal(fl, want), (fraction, fl, want)
        assert int(n.item()) == int(want.sum())
        if fraction == 1.0:
            assert int(want.sum()) == int((sc <= 0.5).sum())       # every kept frame
        a, r = audit.cpu().numpy(), ref.cpu().numpy()
        for b in range(B):
            pr = probes[envs[b][1]]
            sl = slice(int(off[b]), int(off[b]) + pr.out_h * pr.out_w)
            if want[b]:
                assert np.array_equal(a[sl], r[sl]), b
            else:
                assert np.all(a[sl] == -3.0), b
