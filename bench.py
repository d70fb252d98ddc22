"""Benchmark of the batched ultrasound render on GB300.

Default workload: 64 environments on one 256^3 label + HU volume at 0.5 mm,
curvilinear probe 256 lines x 512 samples (60 deg fan), scan-converted to
256 x 256 FP32 frames.  One step = one render of the whole batch (every
stage of the path: slicing, image model, PSF, log compression, scan
conversion) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c2|c1|c3|paper] [--no-plain]

Prints one JSON line.  Under torchrun (N > 1) every rank renders its own
batch (weak scaling, no collective on the data path); the time is the max
over ranks.  ``--impl reference`` times the CPU oracle on the host cores on
the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_01152_gb300 import scene  # noqa: E402

METRIC = "US frames/s on 1 GB300 (physics vs surrogate) at stated error; % HBM roofline"

# Algorithmic ALU work of the physics path, in lane operations (one FP32 /
# INT32 lane op per lane per cycle; an FMA and a shared-memory load count
# once each): ~270 per beam sample (Philox ~60, transcendentals ~15,
# gather and interpolation ~30, the PSF on the reflection impulses and on
# the scatter pattern, 2 x (13 + 21) taps as FMA + load each, the image
# R + E (P (x) T) as one FMA + one load, rest ~60) and ~20 per
# scan-converted output pixel.  Of these, the lateral PSF of both
# (2 x 21 FMA + 2 x 21 loads), the image (2) and the log compression (~5)
# per sample and the per-pixel work belong to pass B of the two-pass path;
# the rest to pass A.
OPS_PER_SAMPLE = 270
OPS_PER_PIXEL = 20
OPS_PER_SAMPLE_PASS_B = 91
# DRAM bytes per launch of the dominant kernel from one ncu capture of the
# current kernel source (absent until captured; dropped when the kernel changes)
KERNEL_DRAM_BYTES = {
    # C3, 512 envs, pass A (16-line groups, as built): 477.79 MB read +
    # 455.38 MB written, one 1-pass capture of the full-size launch
    ("c3_uneven_512env", "split_lines", 16): 933_170_000,
}

# Algorithmic bytes of one launch of the default workload: the union of
# voxels read by the nearest / trilinear footprints of all 64 frames (label
# 1 B + HU 2 B each), the 64 frames written (256 x 256 x 4 B) and the poses
# read (64 x 48 B).  The voxel count comes from the oracle's exact count for
# these poses; the CPU test suite re-derives it.
C2_TOUCHED_VOXELS_VALUE = 3075431
# The same for the 512-env batch of four 512 x 512 x 256 volumes and three
# probes (first step of its random walks), counted per volume and summed.
C3_TOUCHED_VOXELS_VALUE = 18472899


def c2_launch_bytes(B=64):
    return 3 * C2_TOUCHED_VOXELS_VALUE + B * 256 * 256 * 4 + B * 48


def c3_launch_bytes(wl):
    pixels = sum(wl.probes[int(p)].out_w * wl.probes[int(p)].out_h for p in np.asarray(wl.envs)[:, 1])
    return 3 * C3_TOUCHED_VOXELS_VALUE + 4 * pixels + len(wl.envs) * 48


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alu_peak(sms):
    """lane-op/s: SMs x 128 FP32/INT32 lanes x the maximum SM clock"""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "measured clock"
    except Exception:
        mhz, src = 2070.0, "nominal clock"
    return sms * 128 * mhz * 1e6, src


def workload_units(wl):
    """(beam samples, output pixels) of one render of the batch"""
    samples = pixels = 0
    for v, pr in np.asarray(wl.envs):
        p = wl.probes[int(pr)]
        samples += p.n_lines * p.n_samples
        pixels += p.out_w * p.out_h
    return samples, pixels


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            self.out.flush()
            rows = [r.split(",") for r in open(self.out.name).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        finally:
            try:
                os.unlink(self.out.name)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[4:8]):
                if "Active" in v and "Not" not in v:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_workload(name, copies=1):
    """The named workload; `copies` > 1 makes a global batch of that many
    per-rank batches (distinct poses), to be split over the ranks."""
    if name == "c2":
        return scene.workload_c2(64 * copies)
    if name == "c1":
        return scene.workload_c1()
    if name == "paper":
        return scene.workload_paper_replica(100 * copies)
    if name == "surgery3d":
        return scene.workload_surgery3d(128 * copies)
    if name == "c3":
        wl = scene.workload_c3(512 * copies, steps=1)
        wl.poses = wl.poses[0]
        return wl
    if name == "c3v1":
        # C3's probe mix on one of its volumes, 64 envs: a case small enough
        # (about 1.5 GB on the device) for multi-pass profiler captures
        spec = scene.c3_specs()[0]
        lab, hu = scene.make_volume(spec)
        envs = np.stack([np.zeros(64, np.int64), np.arange(64) % 3], axis=1).astype(np.int32)
        poses = scene.random_walk_poses(spec, 64 * copies, 1, 3000)[0]
        return scene.Workload("c3_probe_mix_1vol_64env", [(spec, lab, hu)], scene.c3_probes(),
                              np.tile(envs, (copies, 1)), poses, seed=0x5EED0003)
    raise ValueError(name)


def rank_workload(wl, rank, world):
    """This rank's contiguous, cost-balanced range of a global batch (the
    envs and poses it renders; volumes and probes are shared)."""
    import dataclasses
    from paper_2507_01152_gb300 import shard
    if world == 1:
        return wl, (0, len(wl.envs))
    lo, hi = shard.partition(shard.env_costs(wl.probes, wl.envs), world)[rank]
    sub = dataclasses.replace(wl, envs=wl.envs[lo:hi], poses=wl.poses[lo:hi])
    return sub, (lo, hi)


def cpu_oracle_rate(wl, seconds=10.0, max_frames=None):
    """Frames/s of the CPU oracle as it stands, OpenMP over frames on every
    host core, on a bounded sample of the workload (whole batches repeated
    until ``seconds`` of CPU work)."""
    import oracle
    cores = os.cpu_count() or 1
    vols = [(lab, hu, spec.voxel_mm) for (spec, lab, hu) in wl.volumes]
    B = len(wl.envs)
    n = 0
    t0 = time.perf_counter()
    step = 0
    while True:
        oracle.render_batch(vols, scene.tissue_table(), wl.probes, wl.options, wl.envs, wl.poses, wl.seed, step,
                            n_threads=cores)
        n += B
        step += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_frames and n >= max_frames):
            break
    return n / el, cores, f"{step} x {B}-frame batches of the {wl.name} workload, {el:.1f} s"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, seconds=0.0)
    t0 = time.perf_counter()
    n = 0
    for k in range(args.steps):
        rate, cores, sample = cpu_oracle_rate(wl, seconds=0.0)
        n += len(wl.envs)
    el = time.perf_counter() - t0
    value = n / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "envs": len(wl.envs)},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} batches of {len(wl.envs)} frames (the whole workload)"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def surrogate_speed(sim, wl, B, stream, c=32):
    """frames/s of surrogate inference (slices + forward) on B envs"""
    import torch
    from paper_2507_01152_gb300 import train as T
    from paper_2507_01152_gb300.ussim import make_envs
    spec = wl.volumes[0][0]
    P = torch.from_numpy(scene.dorsal_poses(spec, B, 4242)).cuda()
    envs = np.zeros((B, 2), np.int32)
    ec = make_envs(envs)
    net = T.make_surrogate(c, B, 2e-4, 0)
    x = torch.zeros((B, 256, 256, 8), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((B, 256, 256), device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(2):
            sim.sample_slices(None, P, x, stream=stream, envs_c=ec)
            net.forward(x, y, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = 3
        for _ in range(n):
            sim.sample_slices(None, P, x, stream=stream, envs_c=ec)
            net.forward(x, y, stream=stream)
        b.record(stream)
        b.synchronize()
    net.check(stream)
    ms = a.elapsed_time(b) / n
    net.close()
    return {"value": B / ms * 1e3, "unit": "frames/s", "envs": B, "ms_per_step": ms,
            "tflops": 2 * 10.74e9 * B / ms / 1e9, "base_channels": c,
            "note": "slice sampling + BF16 forward on tcgen05; speed only (weights untrained)",
            "hist_match": hist_match_speed(sim, P, ec, x, stream)}


def hist_match_speed(sim, P, ec, x, stream):
    """CT histogram matching of the surrogate input (per env slice, 4096
    one-HU bins, reference from another synthetic volume): slice sampling
    with and without it, and the standalone matching of B x H x W FP32
    values (algorithmic bytes: two reads of value + mask, one write)"""
    import torch
    # the caller's reference: cumulative counts of a "training CT" (another
    # synthetic volume's integer HU, one-HU bins from -1024)
    other = scene.make_volume(scene.VolumeSpec(96, 96, 96, 0.5, 3, 4321))[1]
    vals = other[other > -1000].astype(np.int64) + 1024
    ref = np.cumsum(np.bincount(np.clip(vals, 0, 4095), minlength=4096)).astype(np.int64)
    B, H, W = x.shape[0], x.shape[1], x.shape[2]
    hu = torch.randn((B, H * W), device="cuda") * 300.0
    mask = torch.ones((B, H * W), dtype=torch.uint8, device="cuda")

    def t(fn, n=5):
        with torch.cuda.stream(stream):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n):
                fn()
            b.record(stream)
            b.synchronize()
        return a.elapsed_time(b) / n

    sim.set_hu_reference(None, 0, 1)
    plain = t(lambda: sim.sample_slices(None, P, x, stream=stream, envs_c=ec))
    sim.set_hu_reference(ref, -1024.0, 1.0)
    matched = t(lambda: sim.sample_slices(None, P, x, stream=stream, envs_c=ec))
    alone = t(lambda: sim.hist_match(hu, mask, hu, stream=stream))
    sim.set_hu_reference(None, 0, 1)
    sim.check(stream)
    peak, which = load_peaks()
    gbs = B * H * W * 14 / alone / 1e6
    return {"slices_ms": plain, "slices_matched_ms": matched, "match_ms": alone, "pixels": B * H * W,
            "match_gbs": gbs, "match_hbm_frac": gbs / peak, "peak_source": which,
            "bytes_per_pixel": 14, "note": "reference: 4096 one-HU bins of another synthetic volume"}


def c5_surrogate_block(args, volumes=None, log=lambda *a: None):
    """The learned surrogate in production (C5), after its training (C4).

    Training: ``args.train_pairs`` fresh physics pairs (curvilinear 256 x 512
    probe on the 256^3 volume, 256 x 256 frames) in batches of
    ``args.train_batch``, every pair rendered on the device in the loop;
    held-out L1 / SSIM on 2048 poses from seeds 1,000,000 on.

    Production step on 1024 envs over the four C3 volumes and the three C3
    probes (a third each): the label / CT slices of every env on one
    256 x 256 grid over its own output field, the surrogate forward, the
    error head, the resize back to each env's frame, then the physics
    fallback for the frames whose predicted L1 gap exceeds the gate and the
    physics audit of a seeded 5% of the frames the gate kept.  The error
    head is fitted on two calibration steps of the same batch (surrogate
    against all-physics, per-frame L1).  Compared with all-physics batched
    and plain per-env renders of the same batch on the same GPU; L1 / SSIM
    of the mixed and surrogate-only frames against the all-physics frames of
    the same step, per probe type."""
    import math as _m
    import torch
    from paper_2507_01152_gb300 import train as T
    from paper_2507_01152_gb300.ussim import Sim, make_envs
    B, G = 1024, 256
    tb = args.train_batch
    steps = max(1, _m.ceil(args.train_pairs / tb))
    t0 = time.perf_counter()
    net, src, hist = T.train(steps, batch=tb, c=32, lr=args.lr, log_every=0, max_batch=B)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    l1_h, ss_h = T.evaluate(net, src, max(1, _m.ceil(2048 / tb)))
    src.sim.close()
    log(f"trained {steps} x {tb} pairs in {train_s:.1f} s; held-out L1 {l1_h:.4f} SSIM {ss_h:.4f}")

    wl = scene.workload_c5(B, steps=3, volumes=volumes)
    dv = [(torch.from_numpy(l).cuda(), torch.from_numpy(h).cuda(), s_.voxel_mm) for (s_, l, h) in wl.volumes]
    sim = Sim(dv, scene.tissue_table(), wl.probes, wl.options)
    envs, ec = wl.envs, make_envs(wl.envs)
    off = sim.frame_layout(envs)
    groups = []                    # (probe, first env, count): contiguous frames of one size
    for p_ in range(3):
        idx = np.nonzero(envs[:, 1] == p_)[0]
        groups.append((p_, int(idx[0]), len(idx)))
    Pw = [torch.from_numpy(np.ascontiguousarray(wl.poses[k])).cuda() for k in range(3)]
    stream = torch.cuda.Stream()
    nf = int(off[-1])
    frames = torch.zeros(nf, device="cuda")
    phys = torch.zeros(nf, device="cuda")
    audit = torch.zeros(nf, device="cuda")
    x = torch.zeros((B, G, G, 8), dtype=torch.bfloat16, device="cuda")
    s256 = torch.zeros((B, G, G), device="cuda")
    pe = torch.zeros(B, device="cuda")
    feat = torch.zeros((B, net.num_features()), device="cuda")
    nr = torch.zeros(1, dtype=torch.int32, device="cuda")
    na = torch.zeros(1, dtype=torch.int32, device="cuda")
    flags = torch.zeros(B, dtype=torch.uint8, device="cuda")
    met = torch.zeros(1 + 2 * B, device="cuda")
    seed = wl.seed
    thr, frac = args.gate_l1, 0.05
    with torch.cuda.stream(stream):
        sim.autotune(envs, Pw[0], phys, None, stream=stream)

    def view(buf, g):
        p_, first, n = g
        pr = wl.probes[p_]
        return buf[int(off[first]):int(off[first]) + n * pr.out_h * pr.out_w].view(n, pr.out_h, pr.out_w)

    def per_frame(a, b):
        """per-frame (L1, SSIM) of frames a against b, env order"""
        l1, ss = np.zeros(B), np.zeros(B)
        for g in groups:
            p_, first, n = g
            net.metrics_hw(view(a, g), view(b, g), met[:1 + 2 * n], stream=stream)
            m = met[:1 + 2 * n].cpu().numpy()
            l1[first:first + n], ss[first:first + n] = m[1:1 + n], m[1 + n:1 + 2 * n]
        return l1, ss

    def surrogate(P):
        sim.sample_slices_grid(None, P, G, G, x, stream=stream, envs_c=ec)
        net.forward(x, s256, stream=stream)
        net.predict_error(B, pe, stream=stream)
        sim.resize_frames(None, s256, frames, stream=stream, envs_c=ec)

    def mixed(P, step):
        surrogate(P)
        sim.render_gated(None, P, seed, step, frames, pe, thr, nr, stream=stream, envs_c=ec)
        sim.render_audit(None, P, seed, step, audit, pe, thr, frac, flags, na, stream=stream, envs_c=ec)

    # error head on two calibration steps (poses of walk steps 1 and 2)
    fs, ys = [], []
    with torch.cuda.stream(stream):
        for k in (1, 2):
            surrogate(Pw[k])
            net.features(B, feat, stream=stream)
            sim.render(None, Pw[k], seed, 900 + k, phys, stream=stream, envs_c=ec)
            l1, _ = per_frame(frames, phys)
            fs.append(feat.cpu().numpy())
            ys.append(l1)
    net.fit_error_head(np.concatenate(fs), np.concatenate(ys), ridge=1e-2)

    def timed(fn, k):
        with torch.cuda.stream(stream):
            for w in range(2):
                fn(100 + w)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(k):
                fn(i)
            b.record(stream)
            b.synchronize()
        return a.elapsed_time(b) / k

    P0 = Pw[0]
    ms_mixed = timed(lambda i: mixed(P0, i), args.c5_steps)
    ms_surr = timed(lambda i: surrogate(P0), args.c5_steps)
    ms_phys = timed(lambda i: sim.render(None, P0, seed, i, phys, stream=stream, envs_c=ec), args.c5_steps)
    ms_plain = timed(lambda i: sim.render_plain(None, P0, seed, i, phys, stream=stream, envs_c=ec), 2)
    # quality of one step against the all-physics render of the same step
    with torch.cuda.stream(stream):
        mixed(P0, 7)
        pe_h = pe.cpu().numpy()
        fl = flags.cpu().numpy().astype(bool)
        n_re = int(nr.item())
        sim.render(None, P0, seed, 7, phys, stream=stream, envs_c=ec)
        mix_l1, mix_ss = per_frame(frames, phys)
        surrogate(P0)
        sur_l1, sur_ss = per_frame(frames, phys)
        aud_l1, _ = per_frame(frames, audit)         # surrogate frames against their audit renders
        stream.synchronize()
    net.check(stream)
    sim.check(stream)
    gated = pe_h > thr
    names = ["linear_128x256", "curvilinear_192x384", "curvilinear_256x512"]
    per_probe = {}
    for (p_, first, n) in groups:
        sl = slice(first, first + n)
        per_probe[names[p_]] = {"envs": n, "rerendered_frac": float(gated[sl].mean()),
                                "mixed_l1": float(mix_l1[sl].mean()), "mixed_ssim": float(mix_ss[sl].mean()),
                                "surrogate_l1": float(sur_l1[sl].mean()), "surrogate_ssim": float(sur_ss[sl].mean())}
    audit_rep = {"fraction": frac, "audited": int(fl.sum()),
                 "pred_abs_err": float(np.abs(pe_h[fl] - aud_l1[fl]).mean()) if fl.any() else None,
                 "true_l1_mean": float(aud_l1[fl].mean()) if fl.any() else None,
                 "missed_over_gate": float((aud_l1[fl] > thr).mean()) if fl.any() else None}
    sim.close()
    net.close()
    return {"workload": wl.name, "envs": B, "grid": f"{G}x{G}", "gate_l1": thr,
            "mixed": {"frames_per_s": B / ms_mixed * 1e3, "ms_per_step": ms_mixed, "rerendered_frac": n_re / B,
                      "l1_vs_physics": float(mix_l1.mean()), "ssim_vs_physics": float(mix_ss.mean()),
                      "meets_gate": bool(mix_l1.mean() <= thr and mix_ss.mean() >= 0.80)},
            "surrogate_only": {"frames_per_s": B / ms_surr * 1e3, "ms_per_step": ms_surr,
                               "l1_vs_physics": float(sur_l1.mean()), "ssim_vs_physics": float(sur_ss.mean()),
                               "tflops": 2 * 10.74e9 * B / ms_surr / 1e9},
            "all_physics_batched": {"frames_per_s": B / ms_phys * 1e3, "ms_per_step": ms_phys},
            "all_physics_plain_per_env": {"frames_per_s": B / ms_plain * 1e3, "ms_per_step": ms_plain},
            "per_probe": per_probe, "audit": audit_rep,
            "training": {"pairs": steps * tb, "batch": tb, "steps": steps, "seconds": train_s,
                         "heldout_poses": max(1, _m.ceil(2048 / tb)) * tb, "heldout_l1": l1_h, "heldout_ssim": ss_h,
                         "loss_first_last": [hist[0][1], hist[-1][1]]}}


def run_mixed(args):
    """The C4 training and C5 production step alone, as one JSON line."""
    import torch
    from paper_2507_01152_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    blk = c5_surrogate_block(args, log=lambda m: print(m, file=sys.stderr, flush=True))
    line = {"metric": METRIC, "value": blk["mixed"]["frames_per_s"], "unit": "frames/s", "n_gpus": 1,
            "steps": args.c5_steps, "warmup": 2, "ms_per_step": blk["mixed"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": blk["workload"], "envs": blk["envs"],
                       "gate": f"physics re-render where predicted L1 > {blk['gate_l1']}; 5% physics audit"},
            "surrogate": blk}
    print(json.dumps(line), flush=True)


def run_recon(args):
    """Bone-surface task step (Task 2; App. C): 128 envs with the 200 x 150
    linear probe on the 256^3 volume; every step renders the batch, adds the
    kept bone-surface points (20% missing) to each env's reconstruction and
    voxelizes the reconstructions to 40^3 observations at 3 mm in the probe
    frame.  Reports env steps per second (device time, L2 flushed)."""
    import torch
    from paper_2507_01152_gb300 import build
    from paper_2507_01152_gb300.ussim import Sim, make_envs
    build.build()
    torch.cuda.set_device(0)
    spec = scene.c2_spec()
    lab, hu = scene.make_volume(spec)
    B, T = 128, args.steps + args.warmup + 1
    probe = scene.linear_probe(150, 200, 100.0, 0.5)
    walk = scene.random_walk_poses(spec, B, T, 2005)
    envs = np.zeros((B, 2), np.int32)
    sim = Sim([(torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), spec.voxel_mm)], scene.tissue_table(),
              [probe], scene.Options())
    ec = make_envs(envs)
    off = sim.frame_layout(envs)
    frames = torch.empty(int(off[-1]), device="cuda")
    words, cap = sim.recon_words(), 1 << 16
    bm = torch.zeros((B, words), dtype=torch.int32, device="cuda")
    pts = torch.zeros((B, cap), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(B, dtype=torch.int32, device="cuda")
    obs = torch.zeros((B, 40, 40, 40), dtype=torch.uint8, device="cuda")
    P = torch.from_numpy(np.ascontiguousarray(walk, np.float32)).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        sim.autotune(envs, P[0], frames, None, stream=st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    tr = tu = to = 0.0
    with torch.cuda.stream(st):
        for t in range(T):
            flush.zero_()
            ev[0].record(st)
            sim.render(None, P[t], 7, t, frames, stream=st, envs_c=ec)
            ev[1].record(st)
            sim.recon_update(envs, P[t], 7, t, 4, 0.2, bm, pts, cnt, stream=st, envs_c=ec)
            ev[2].record(st)
            sim.recon_observe(envs, P[t], pts, cnt, obs, stream=st, envs_c=ec)
            ev[3].record(st)
            ev[3].synchronize()
            if t > args.warmup:
                tr += ev[0].elapsed_time(ev[1])
                tu += ev[1].elapsed_time(ev[2])
                to += ev[2].elapsed_time(ev[3])
    sim.check(st)
    K = T - args.warmup - 1
    ms = (tr + tu + to) / K
    line = {"metric": METRIC, "value": B / ms * 1e3, "unit": "frames/s", "n_gpus": 1, "steps": K,
            "warmup": args.warmup + 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "bone_surface_task_128env_linear_200x150_recon40", "envs": B,
                       "frame": "one env step: render + reconstruction update + 40^3 observation",
                       "l2": "flushed between timed steps (256 MB write)", "tuning": sim.get_tuning()},
            "breakdown_ms": {"render": tr / K, "recon_update": tu / K, "recon_observe": to / K},
            "reconstructed_voxels_per_env_after": float(cnt.float().mean()),
            "occupied_obs_voxels_per_env": float(obs.float().sum()) / B}
    print(json.dumps(line), flush=True)
    sim.close()


def run_ours(args):
    import torch
    from paper_2507_01152_gb300 import build
    from paper_2507_01152_gb300.ussim import Sim, make_envs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()

    from paper_2507_01152_gb300 import shard
    # weak scaling: a global batch of `world` per-rank batches, split into
    # contiguous cost-balanced ranges (no collective on the data path)
    if args.workload == "c1":      # a single environment: every rank renders its own copy
        wl = make_workload("c1")
    else:
        wl, _ = rank_workload(make_workload(args.workload, world), rank, world)
    if args.speckle == "anchored":   # fixed two-scale scatter maps over the volume (0.25 mm cells)
        import dataclasses
        wl = dataclasses.replace(wl, options=dataclasses.replace(wl.options, speckle_anchor=1, speckle_levels=2,
                                                                 speckle_cell_mm=0.25))
    wl3 = None
    if args.workload == "surgery3d":
        # the timed render sweeps each probe over its elevation slices on the
        # device (us_sim_render_3d); the other measurements use the expanded
        # batch of 2-D slices (same kernels, host-swept poses)
        import dataclasses
        E, pitch = scene.SURGERY3D_SLICES, scene.SURGERY3D_PITCH_MM
        wl3 = wl
        from paper_2507_01152_gb300 import ussim
        p3 = torch.from_numpy(np.ascontiguousarray(wl.poses, np.float32)).cuda()
        swept = torch.empty((len(wl.poses) * E, 3, 4), dtype=torch.float32, device="cuda")
        ussim.sweep_poses(p3, E, pitch, swept)
        torch.cuda.synchronize()
        wl = dataclasses.replace(wl, envs=np.repeat(wl.envs, E, axis=0), poses=swept.cpu().numpy())
    B = len(wl.envs)
    vols = [(torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), spec.voxel_mm) for (spec, lab, hu) in wl.volumes]
    sim = Sim(vols, scene.tissue_table(), wl.probes, wl.options)
    envs_c = make_envs(wl.envs)
    off = sim.frame_layout(wl.envs)
    stream = torch.cuda.Stream()
    poses = torch.from_numpy(np.ascontiguousarray(wl.poses, np.float32)).cuda()
    frames = torch.empty(int(off[-1]), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    seed = shard.rank_seed(wl.seed, rank)

    def timed(fn, steps, warmup):
        with torch.cuda.stream(stream):
            for w in range(warmup):
                fn(1000 + w)
            stream.synchronize()
            times = []
            for k in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn(k)
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b) / 1000.0)
        return times

    # launch shape from the autotuner (cached per GPU / probe set / batch), graph replay on
    tune_cache = os.path.join(build.BUILD, "autotune.txt")
    with torch.cuda.stream(stream):
        sim.autotune(wl.envs, poses, frames, tune_cache, stream=stream)
    tuning = sim.get_tuning()
    sim.set_tuning(tuning["cluster_size"], tuning["warps_per_cta"], 1, tuning["persistent"], tuning["wedge_lines"])
    tuning = sim.get_tuning()
    two_grids = tuning["cluster_size"] == 1 and not tuning["persistent"]
    render = lambda k: sim.render(None, poses, seed, k, frames, stream=stream, envs_c=envs_c)
    if wl3 is not None:
        poses3 = torch.from_numpy(np.ascontiguousarray(wl3.poses, np.float32)).cuda()
        render = lambda k: sim.render_3d(wl3.envs, poses3, scene.SURGERY3D_SLICES, scene.SURGERY3D_PITCH_MM, seed, k,
                                         frames, stream=stream)
    if wl3 is None:
        # the timed form (graph replays of the tuned shape) must render what
        # the plain per-env kernels render: two replays checked bit for bit
        check = torch.empty_like(frames)
        for k in (11, 12):
            render(k)
            sim.render_plain(None, poses, seed, k, check, stream=stream, envs_c=envs_c)
            stream.synchronize()
            if not torch.equal(frames, check):
                raise RuntimeError(f"tuned render {tuning} differs from the plain kernels (step {k})")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = timed(render, args.steps, args.warmup)
    torch.cuda.synchronize()
    total = sum(times)
    sim.check(stream)
    total, frames_all = shard.reduce_timing(total, B * args.steps, dist, device="cuda")
    if dist is not None:
        dist.barrier()
    value = frames_all / total
    kernel_s = total / args.steps           # device time of one render step (all its kernels)

    # plain per-environment form on the same batch (comparison)
    plain = None
    if not args.no_plain:
        ptimes = timed(lambda k: sim.render_plain(None, poses, seed, k, frames, stream=stream, envs_c=envs_c),
                       max(3, args.steps // 4), 2)
        plain = {"value": B * len(ptimes) / sum(ptimes), "unit": "frames/s",
                 "ms_per_step": 1000 * sum(ptimes) / len(ptimes), "launches_per_step": 5 * B}

    # end to end through the host-buffer entry point: pose copy in, frames out
    host_poses = torch.from_numpy(np.ascontiguousarray(wl.poses, np.float32)).pin_memory().numpy()
    host_frames = torch.empty(int(off[-1]), dtype=torch.float32).pin_memory().numpy()
    for w in range(2):
        sim.render_host(None, host_poses, seed, 5000 + w, host_frames, stream=stream, envs_c=envs_c)
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps)
    for k in range(e2e_steps):
        sim.render_host(None, host_poses, seed, 6000 + k, host_frames, stream=stream, envs_c=envs_c)
    e2e_el, e2e_frames = shard.reduce_timing(time.perf_counter() - t0, B * e2e_steps, dist, device="cuda")
    e2e = {"value": e2e_frames / e2e_el, "unit": "frames/s", "h2d_bytes_per_step": int(host_poses.nbytes),
           "d2h_bytes_per_step": int(host_frames.nbytes)}

    # per-kernel durations of the same render (events around each kernel on
    # the launching stream, L2 flushed before every call)
    kms = []
    with torch.cuda.stream(stream):
        for k in range(max(5, args.steps // 2)):
            flush.zero_()
            kms.append(sim.render_timed(None, poses, seed, 7000 + k, frames, stream=stream, envs_c=envs_c))
    kavg = [sum(x[i] for x in kms) / len(kms) for i in range(len(kms[0]))]
    names = (["split_lines", "split_image"] if two_grids
             else ["split_persist"] if tuning["cluster_size"] == 1 else ["fused_render"])
    dom = max(range(len(kavg)), key=lambda i: kavg[i])
    samples, pixels = workload_units(wl)
    if len(names) == 1:
        ops = OPS_PER_SAMPLE * samples + OPS_PER_PIXEL * pixels
    elif dom == 0:
        ops = (OPS_PER_SAMPLE - OPS_PER_SAMPLE_PASS_B) * samples
    else:
        ops = OPS_PER_SAMPLE_PASS_B * samples + OPS_PER_PIXEL * pixels
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    apeak, asrc = alu_peak(sms)
    achieved = ops / (kavg[dom] / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": apeak / 1e12, "unit": "Tlane-op/s",
                "frac": achieved * 1e12 / apeak,
                "traffic": KERNEL_DRAM_BYTES.get((wl.name if args.speckle == "beam" else None, names[dom],
                                                  tuning["warps_per_cta"])),
                "kernel": names[dom], "kernel_ms": kavg[dom], "kernels_ms": dict(zip(names, kavg)),
                "lane_ops_per_launch": ops, "peak_source": f"{sms} SMs x 128 lanes x {asrc}"}
    alg_bytes = None
    if world == 1 and args.workload == "c2":
        alg_bytes = c2_launch_bytes(B)
    elif world == 1 and args.workload == "c3":
        alg_bytes = c3_launch_bytes(wl)
    if alg_bytes is not None:
        peak, which = load_peaks()
        hb = alg_bytes / kernel_s / 1e9
        roofline["hbm"] = {"achieved": hb, "peak": peak, "unit": "GB/s", "frac": hb / peak, "peak_source": which,
                           "bytes_per_step": alg_bytes, "scope": "whole render step",
                           "bytes": "union of touched voxels (label 1 B + HU 2 B, the oracle's exact count) + "
                                    "frames written + poses"}

    # the learned surrogate: trained at the C4 size, then the C5 production
    # step (surrogate + error gate + physics fallback + audit) beside
    # all-physics on the same GPU
    surrogate = None
    if args.workload == "c2" and not args.no_surrogate:
        # surrogate inference throughput at 512 envs (speed only: the cost
        # of a forward pass does not depend on the weights)
        surrogate = surrogate_speed(sim, wl, 512, stream)
    if args.workload == "c3" and world == 1 and not args.no_surrogate:
        sim.close()
        sim = None
        surrogate = c5_surrogate_block(args, volumes=wl.volumes)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_rate(wl, seconds=args.cpu_seconds)
        cpu = {"value": rate, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name + ("_anchored_speckle" if args.speckle == "anchored" else ""),
                           "envs_per_gpu": B, "l2": "flushed between timed steps (256 MB write)",
                           **({"volumetric_images_per_s": value / scene.SURGERY3D_SLICES,
                               "frame": "one 50 x 37 elevation slice (5 per volumetric image)"}
                              if wl3 is not None else {}),
                           "path": ("two-pass batched kernels" if two_grids
                                    else "two-pass path in one persistent grid" if tuning["cluster_size"] == 1
                                    else "persistent cluster kernel") + ", CUDA graph replay, autotuned",
                           "tuning": tuning,
                           "parallelism": f"{world} ranks, contiguous cost-balanced env shards, no collective"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * (2 if two_grids else 1),
                "plain": plain, "surrogate": surrogate, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c1", "paper", "surgery3d", "recon", "mixed",
                                                         "c3v1"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--train-pairs", type=int, default=200_000, help="surrogate training pairs (C4: 200k)")
    ap.add_argument("--train-batch", type=int, default=256, help="surrogate training batch (C4: 256)")
    ap.add_argument("--c5-steps", type=int, default=10, help="timed steps of the C5 production step")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--gate-l1", type=float, default=0.05)
    ap.add_argument("--speckle", default="beam", choices=["beam", "anchored"],
                    help="scatter maps keyed by beam sample (default) or fixed over the volume")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "recon":
        run_recon(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
