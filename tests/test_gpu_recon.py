"""Reconstruction observation (Task 2) on the GPU against the oracle: the
reconstructed voxel sets after several steps and the 40^3 observations,
exactly."""
import numpy as np
import pytest

import oracle
from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_reconstruction_and_observation_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    from simhelp import gpu_sim
    build.build()
    spec = scene.c1_spec()
    lab, hu = scene.make_volume(spec)
    probes = [scene.linear_probe(150, 200, 100.0, 0.5), scene.curvilinear_probe(64, 128, 80.0, 60.0, 40.0, 64, 64)]
    B, steps = 6, 6
    walk = scene.random_walk_poses(spec, B, steps, 77)            # [steps][B][3][4]
    envs = np.stack([np.zeros(B), np.arange(B) % 2], axis=1).astype(np.int32)
    wl = scene.Workload("recon", [(spec, lab, hu)], probes, envs, walk[0], seed=0x5EED0007)
    sim = gpu_sim(wl)
    words = sim.recon_words()
    assert words == (128 ** 3 + 31) // 32
    cap = 1 << 16
    bm = torch.zeros((B, words), dtype=torch.int32, device="cuda")
    pts = torch.zeros((B, cap), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(B, dtype=torch.int32, device="cuda")
    obs = torch.zeros((B, 40, 40, 40), dtype=torch.uint8, device="cuda")
    rec = [np.zeros(lab.shape, np.uint8) for _ in range(B)]
    for t in range(steps):
        P = torch.from_numpy(np.ascontiguousarray(walk[t], np.float32)).cuda()
        sim.recon_update(envs, P, wl.seed, t, 4, 0.2, bm, pts, cnt)
        for b in range(B):
            oracle.recon_update(lab, hu, spec.voxel_mm, probes[envs[b][1]], walk[t][b], b, wl.seed, t, 4, 0.2, rec[b])
    P = torch.from_numpy(np.ascontiguousarray(walk[-1], np.float32)).cuda()
    sim.recon_observe(envs, P, pts, cnt, obs)
    torch.cuda.synchronize()
    sim.check()
    bits = bm.cpu().numpy().view(np.uint32)
    c = cnt.cpu().numpy()
    pl = pts.cpu().numpy()
    o = obs.cpu().numpy()
    total = 0
    for b in range(B):
        want = np.flatnonzero(rec[b].reshape(-1))
        got_bits = np.flatnonzero(np.unpackbits(bits[b].view(np.uint8), bitorder="little")[:lab.size])
        assert np.array_equal(got_bits, want), b
        assert c[b] == len(want) and np.array_equal(np.sort(pl[b, :c[b]]), want)
        assert np.array_equal(o[b], oracle.recon_observe(rec[b], spec.voxel_mm, walk[-1][b])), b
        total += len(want)
    assert total > 20 and o.sum() > 0                             # the probes do see bone
