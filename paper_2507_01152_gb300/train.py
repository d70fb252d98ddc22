"""Training and evaluation of the learned surrogate on pairs the physics
path renders on the GPU (every step of data generation, forward, loss,
backward and update runs in libussim's kernels; this module only
sequences the calls and moves scalars to the host for logging).

Pairs: seeded dorsal poses on the 256^3 spine-like volume; input = the
label / HU slice on the 256 x 256 output grid of the curvilinear probe
(``us_sim_sample_slices``), target = the physics frame (``us_sim_render``)
of the same pose, speckle keyed by the pose's seed.  Training poses are
drawn from seeds 0, 1, ...; held-out poses from seeds 1_000_000 + k.
"""
from __future__ import annotations

import time

import numpy as np

from . import scene

HELD_OUT_SEED = 1_000_000


class PairSource:
    """Renders (input slice, physics frame) batches on the GPU."""

    def __init__(self, batch: int, spec=None, probe=None, seed: int = 0x5EED0004, tuning=None):
        import torch
        from .ussim import Sim, make_envs
        self.torch = torch
        self.spec = spec or scene.c2_spec()
        lab, hu = scene.make_volume(self.spec)
        self.probe = probe or scene.curvilinear_probe()
        self.vol = (torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), self.spec.voxel_mm)
        self.sim = Sim([self.vol], scene.tissue_table(), [self.probe], scene.Options())
        self.B = batch
        self.envs = np.zeros((batch, 2), np.int32)
        self.envs_c = make_envs(self.envs)
        self.seed = seed
        H, W = self.probe.out_h, self.probe.out_w
        self.x = torch.zeros((batch, H, W, 8), dtype=torch.bfloat16, device="cuda")
        self.y = torch.zeros((batch, H, W), dtype=torch.float32, device="cuda")
        self.poses = torch.zeros((batch, 3, 4), dtype=torch.float32, device="cuda")

    def batch(self, pose_seed: int, step: int, stream=None):
        """fill self.x / self.y for B poses drawn from ``pose_seed``"""
        P = scene.dorsal_poses(self.spec, self.B, pose_seed)
        self.poses.copy_(self.torch.from_numpy(P))
        self.sim.render(None, self.poses, self.seed, step, self.y, stream=stream, envs_c=self.envs_c)
        self.sim.sample_slices(None, self.poses, self.x, stream=stream, envs_c=self.envs_c)
        return self.x, self.y


def gate_samples(net, src: PairSource, n_batches: int, first_seed: int = HELD_OUT_SEED + 1000):
    """(features, true per-frame L1) of the surrogate against physics on
    ``n_batches`` batches of poses (for fitting the error head)"""
    torch = src.torch
    F = net.num_features()
    feat = torch.zeros((src.B, F), device="cuda")
    out = torch.zeros(1 + 2 * src.B, device="cuda")
    pred = torch.zeros_like(src.y)
    fs, ys = [], []
    for k in range(n_batches):
        x, y = src.batch(first_seed + k, first_seed + k)
        net.forward(x, pred)
        net.features(src.B, feat)
        net.metrics(pred, y, out)
        fs.append(feat.cpu().numpy())
        ys.append(out[1:1 + src.B].cpu().numpy())
    return np.concatenate(fs), np.concatenate(ys)


def mixed_step(sim, net, poses, seed, step, x, frames, err_pred, threshold, n_rendered, stream=None, envs_c=None):
    """One production step: surrogate frames for every env, physics
    re-render of the frames whose predicted error exceeds ``threshold``."""
    B = poses.shape[0]
    sim.sample_slices(None, poses, x, stream=stream, envs_c=envs_c)
    net.forward(x, frames, stream=stream)
    net.predict_error(B, err_pred, stream=stream)
    sim.render_gated(None, poses, seed, step, frames, err_pred, threshold, n_rendered, stream=stream, envs_c=envs_c)


def make_surrogate(c: int, batch: int, lr: float, seed: int, H=256, W=256):
    from .ussim import Surrogate
    off, size, fan = Surrogate.segments(c, H, W)
    return Surrogate(c, H, W, batch, scene.surrogate_init(size, fan, seed), lr=lr)


def evaluate(net, src: PairSource, n_batches: int = 2):
    """mean held-out L1 / SSIM of the surrogate against physics"""
    torch = src.torch
    out = torch.zeros(1 + 2 * src.B, device="cuda")
    pred = torch.zeros_like(src.y)
    l1, ss = [], []
    for k in range(n_batches):
        x, y = src.batch(HELD_OUT_SEED + k, HELD_OUT_SEED + k)
        net.forward(x, pred)
        net.metrics(pred, y, out)
        o = out.cpu().numpy()
        l1.append(o[1:1 + src.B])
        ss.append(o[1 + src.B:])
    return float(np.mean(np.concatenate(l1))), float(np.mean(np.concatenate(ss)))


def train(steps: int, batch: int = 256, c: int = 32, lr: float = 2e-4, seed: int = 0, log_every: int = 50,
          eval_batches: int = 2, log=print, probe=None, max_batch=None):
    """Train for ``steps`` steps of ``batch`` fresh pairs; returns (net,
    source, history).  ``max_batch`` sizes the network's buffers for later
    inference on larger batches."""
    torch = __import__("torch")
    src = PairSource(batch, probe=probe)
    net = make_surrogate(c, max(batch, max_batch or 0), lr, seed, src.probe.out_h, src.probe.out_w)
    loss = torch.zeros(1 + 2 * batch, device="cuda")
    hist = []
    t0 = time.perf_counter()
    for s in range(steps):
        x, y = src.batch(s, s)
        net.train_step(x, y, loss, update=True)
        logged = log_every and s % log_every == 0
        if logged or s == 0 or s == steps - 1:
            l = float(loss[0])
            hist.append((s, l))
            if log_every:
                log(f"step {s} loss {l:.4f} ({time.perf_counter() - t0:.1f} s)")
    net.check()
    return net, src, hist
