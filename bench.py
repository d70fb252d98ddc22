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

# Algorithmic bytes of one launch of the default workload: the union of
# voxels read by the nearest / trilinear footprints of all 64 frames (label
# 1 B + HU 2 B each), the 64 frames written (256 x 256 x 4 B) and the poses
# read (64 x 48 B).  The voxel count comes from the oracle's exact count for
# these poses; the CPU test suite re-derives it.
C2_TOUCHED_VOXELS_VALUE = 3075431


def c2_launch_bytes(B=64):
    return 3 * C2_TOUCHED_VOXELS_VALUE + B * 256 * 256 * 4 + B * 48


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def make_workload(name):
    if name == "c2":
        return scene.workload_c2(64)
    if name == "c1":
        return scene.workload_c1()
    if name == "paper":
        return scene.workload_paper_replica(100)
    if name == "c3":
        wl = scene.workload_c3(512, steps=1)
        wl.poses = wl.poses[0]
        return wl
    raise ValueError(name)


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

    wl = make_workload(args.workload)
    B = len(wl.envs)
    vols = [(torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), spec.voxel_mm) for (spec, lab, hu) in wl.volumes]
    sim = Sim(vols, scene.tissue_table(), wl.probes, wl.options)
    envs_c = make_envs(wl.envs)
    off = sim.frame_layout(wl.envs)
    stream = torch.cuda.Stream()
    poses = torch.from_numpy(np.ascontiguousarray(wl.poses, np.float32)).cuda()
    frames = torch.empty(int(off[-1]), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    seed = wl.seed + 7919 * rank

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
    sim.set_tuning(tuning["cluster_size"], tuning["warps_per_cta"], 1)
    tuning = sim.get_tuning()
    render = lambda k: sim.render(None, poses, seed, k, frames, stream=stream, envs_c=envs_c)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = timed(render, args.steps, args.warmup)
    torch.cuda.synchronize()
    total = sum(times)
    sim.check(stream)
    if dist is not None:
        t = torch.tensor([total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
        dist.barrier()
    value = B * args.steps * world / total
    kernel_s = total / args.steps           # one fused launch per step: the event time is the kernel's

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
    e2e_el = time.perf_counter() - t0
    e2e = {"value": B * e2e_steps / e2e_el * world, "unit": "frames/s", "h2d_bytes_per_step": int(host_poses.nbytes),
           "d2h_bytes_per_step": int(host_frames.nbytes)}

    roofline = None
    if args.workload == "c2":
        peak, which = load_peaks()
        achieved = c2_launch_bytes(B) / kernel_s / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "peak_source": which, "kernel": "fused_render",
                    "bytes_per_launch": c2_launch_bytes(B)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_rate(wl, seconds=args.cpu_seconds)
        cpu = {"value": rate, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "envs_per_gpu": B, "l2": "flushed between timed steps (256 MB write)",
                           "path": "fused persistent cluster kernel, CUDA graph replay",
                           "tuning": tuning, "parallelism": f"replicas{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "plain": plain, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "paper"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
