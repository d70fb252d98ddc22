"""Shared helpers for the tests: move a workload to the GPU, render through
the C ABI, render the same batch with the oracle, compare."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2507_01152_gb300 import scene


def gpu_sim(wl, options=None, table=None):
    import torch
    from paper_2507_01152_gb300.ussim import Sim
    vols = []
    for (spec, lab, hu) in wl.volumes:
        vols.append((torch.from_numpy(np.ascontiguousarray(lab)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(hu)).cuda(), spec.voxel_mm))
    return Sim(vols, table or scene.tissue_table(), wl.probes, options or wl.options)


def render_gpu(sim, envs, poses, seed, step, path=0, debug=True):
    """Render through us_sim_render_debug (path 0 fused, 1 plain) or
    us_sim_render / us_sim_render_plain (debug=False).  Returns a list of
    per-env dicts of numpy arrays."""
    import torch
    B = len(envs)
    off = sim.frame_layout(envs)
    boff = sim.beam_layout(envs)
    P = torch.from_numpy(np.ascontiguousarray(poses, np.float32).reshape(B, 3, 4)).cuda()
    frames = torch.full((int(off[-1]),), -7.0, dtype=torch.float32, device="cuda")
    out = []
    if debug:
        nb = int(boff[-1])
        env = torch.full((nb,), -7.0, dtype=torch.float32, device="cuda")
        logi = torch.full((nb,), -7.0, dtype=torch.float32, device="cuda")
        nn = torch.full((nb,), -9, dtype=torch.int32, device="cuda")
        lab = torch.full((nb,), 255, dtype=torch.uint8, device="cuda")
        sim.render_debug(envs, P, seed, step, frames, env, logi, nn, lab, path=path)
        torch.cuda.synchronize()
        env, logi, nn, lab = env.cpu().numpy(), logi.cpu().numpy(), nn.cpu().numpy(), lab.cpu().numpy()
    else:
        (sim.render if path == 0 else sim.render_plain)(envs, P, seed, step, frames)
        torch.cuda.synchronize()
    fr = frames.cpu().numpy()
    for b in range(B):
        pr = sim.probes[int(envs[b][1])]
        d = {"frame": fr[off[b]:off[b] + pr.out_h * pr.out_w].reshape(pr.out_h, pr.out_w)}
        if debug:
            sl = slice(int(boff[b]), int(boff[b + 1]))
            shp = (pr.n_lines, pr.n_samples)
            d.update(envelope=env[sl].reshape(shp), logimg=logi[sl].reshape(shp),
                     nn_index=nn[sl].reshape(shp), label=lab[sl].reshape(shp))
        out.append(d)
    return out


def render_oracle(wl, envs, poses, seed, step, which, options=None, table=None):
    """Oracle render of the envs listed in ``which`` (env index b keeps its
    batch position for the noise counter)."""
    res = {}
    for b in which:
        v, p = int(envs[b][0]), int(envs[b][1])
        spec, lab, hu = wl.volumes[v]
        res[b] = oracle.render_frame(lab, hu, spec.voxel_mm, table or scene.tissue_table(), wl.probes[p],
                                     options or wl.options, poses[b], env=b, seed=seed, step=step)
    return res


def compare(g, o, probe, frame_tol=1e-3):
    """Parity bar: labels and nearest indices bit-exact; pre-log envelope
    within 1e-4 of the frame's maximum; log image within 1e-3 where the
    oracle envelope is at least 1e-3 E0 (0.02 elsewhere); final frame
    within ``frame_tol``."""
    msgs = []
    if "nn_index" in g:
        if not np.array_equal(g["nn_index"], o["nn_index"]):
            msgs.append(f"nn_index mismatch at {np.argwhere(g['nn_index'] != o['nn_index'])[:5].tolist()}")
        if not np.array_equal(g["label"], o["label"]):
            msgs.append("label mismatch")
        scale = np.abs(o["envelope"]).max()
        env_err = np.abs(g["envelope"] - o["envelope"]).max() / max(scale, 1e-300)
        if env_err > 1e-4:
            msgs.append(f"envelope rel err {env_err:.3e}")
        good = o["envelope"] >= 1e-3 * probe.e0
        dy = np.abs(g["logimg"] - o["logimg"])
        if good.any() and dy[good].max() > 1e-3:
            msgs.append(f"logimg err (conditioned) {dy[good].max():.3e}")
        if dy.max() > 0.02:
            msgs.append(f"logimg err {dy.max():.3e}")
    df = np.abs(g["frame"] - o["frame"]).max()
    if df > frame_tol:
        msgs.append(f"frame err {df:.3e}")
    return msgs
