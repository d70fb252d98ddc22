"""Timing of single operators on the GPU (CUDA events, after warm-up).

    python -m paper_2507_01152_gb300.opbench fwd|dgrad|wgrad B H Cin Cout [stride] [reps]
    python -m paper_2507_01152_gb300.opbench hist B H [reps]
    python -m paper_2507_01152_gb300.opbench surrogate B [reps]
    python -m paper_2507_01152_gb300.opbench train B [reps]

fwd / dgrad / wgrad: one 3x3 convolution pass of the tcgen05 implicit GEMM
on B images of H x H pixels (input grid), NHWC BF16 activations with random
values, Cin -> Cout channels; prints the time per call and the rate in
TFLOP/s (2 x 9 x Cin x Cout multiply-adds per output pixel).

surrogate: the whole surrogate forward (base 32 channels, 256 x 256
frames) on B random input slices; prints the time per call, frames/s and
TFLOP/s (2 x 10.74 G multiply-adds per frame).

train: one surrogate training step (forward, L1 + 1 - SSIM, full backward,
Adam) on B random slices and targets; prints the time per step.

hist: CT histogram matching (us_sim_hist_match) of B images of H x H FP32
values (normal, 300 HU spread, every pixel considered) to a reference of
4096 one-HU bins; prints the time per call and the rate in GB/s of
algorithmic bytes (value and mask read twice, value written: 14 B per
pixel)."""
from __future__ import annotations

import sys


def conv3x3(kind: str, B: int, H: int, Cin: int, Cout: int, stride: int = 1, reps: int = 10):
    import torch
    from . import build
    from .ussim import op
    build.build()
    dev = "cuda"
    bf = torch.bfloat16
    Ho = (H - 1) // stride + 1
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    g = torch.Generator(device=dev).manual_seed(1)
    x = torch.randn(B, H, H, Cin, device=dev, generator=g).relu().to(bf)
    dy = torch.randn(B, Ho, Ho, Cout, device=dev, generator=g).to(bf)
    if kind == "fwd":
        w = (torch.randn(Cout, 3, 3, Cin, device=dev, generator=g) * 0.05).to(bf)
        b = torch.zeros(Cout, device=dev)
        y = torch.empty(B, Ho, Ho, Cout, device=dev, dtype=bf)
        call = lambda: op("us_conv3x3_fwd", x, Cin, 0, w, b, y, Cout, 0, B, H, H, Cin, Cout, stride, 1, err)
    elif kind == "dgrad":
        wd = (torch.randn(Cin, 9 * Cout, device=dev, generator=g) * 0.05).to(bf)
        dx = torch.empty(B, H, H, Cin, device=dev, dtype=bf)
        call = lambda: op("us_conv3x3_dgrad", dy, Cout, 0, wd, x, Cin, 0, dx, Cin, 0, 0, B, H, H, Cin, Cout, stride, err)
    elif kind == "wgrad":
        gw = torch.zeros(9 * Cin, Cout, device=dev)
        call = lambda: op("us_conv3x3_wgrad", x, Cin, 0, dy, Cout, 0, gw, B, H, H, Cin, Cout, stride, err)
    else:
        raise ValueError(kind)
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        call()
    e.record()
    e.synchronize()
    ms = a.elapsed_time(e) / reps
    if int(err.item()):
        raise RuntimeError(f"device error word {int(err.item())}")
    flop = 2.0 * B * Ho * Ho * 9 * Cin * Cout
    return ms, flop / ms / 1e9


def hist_match(B: int, H: int, reps: int = 10):
    import numpy as np
    import torch
    from . import build, scene
    from .ussim import Sim
    build.build()
    spec = scene.VolumeSpec(32, 32, 32, 1.0, 1, 7)
    lab, hu = scene.make_volume(spec)
    sim = Sim([(torch.from_numpy(lab).cuda(), torch.from_numpy(hu).cuda(), 1.0)], scene.tissue_table(),
              [scene.linear_probe(16, 32, 30.0, 1.0)])
    # reference: a CT-like spread of integer HU, one-HU bins from -1024
    rng = np.random.default_rng(3)
    vals = np.clip(np.round(rng.gamma(2.5, 150.0, 200000) - 500.0).astype(np.int64) + 1024, 0, 4095)
    sim.set_hu_reference(np.cumsum(np.bincount(vals, minlength=4096)), -1024.0, 1.0)
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn((B, H * H), device="cuda", generator=g) * 300.0
    m = torch.ones((B, H * H), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        sim.hist_match(x, m, y)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        sim.hist_match(x, m, y)
    e.record()
    e.synchronize()
    sim.check()
    ms = a.elapsed_time(e) / reps
    sim.close()
    return ms, B * H * H * 14 / ms / 1e6


def surrogate_forward(B: int, reps: int = 5, c: int = 32, H: int = 256):
    """the whole surrogate forward (c base channels, H x H frames) on B
    random BF16 input slices: ms per call, frames/s, TFLOP/s (2 x the
    network's multiply-adds)"""
    import numpy as np
    import torch
    from . import build, scene
    from .ussim import Surrogate
    build.build()
    off, size, fan = Surrogate.segments(c, H, H)
    net = Surrogate(c, H, H, B, scene.surrogate_init(size, fan, 0))
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.rand((B, H, H, 8), device="cuda", generator=g).to(torch.bfloat16)
    y = torch.empty((B, H, H), device="cuda")
    for _ in range(2):
        net.forward(x, y)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        net.forward(x, y)
    e.record()
    e.synchronize()
    net.check()
    ms = a.elapsed_time(e) / reps
    macs = 10.74e9 * (c / 32) ** 2 * (H / 256) ** 2
    net.close()
    return ms, B / ms * 1e3, 2 * macs * B / ms / 1e9


def surrogate_train(B: int, reps: int = 3, c: int = 32, H: int = 256):
    """one training step of the surrogate (forward, L1 + 1 - SSIM, full
    backward, Adam) on B random BF16 slices and targets: ms per step"""
    import torch
    from . import build, scene
    from .ussim import Surrogate
    build.build()
    off, size, fan = Surrogate.segments(c, H, H)
    net = Surrogate(c, H, H, B, scene.surrogate_init(size, fan, 0))
    g = torch.Generator(device="cuda").manual_seed(2)
    x = torch.rand((B, H, H, 8), device="cuda", generator=g).to(torch.bfloat16)
    y = torch.rand((B, H, H), device="cuda", generator=g)
    loss = torch.zeros(1 + 2 * B, device="cuda")
    for _ in range(2):
        net.train_step(x, y, loss, update=True)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        net.train_step(x, y, loss, update=True)
    e.record()
    e.synchronize()
    net.check()
    net.close()
    return a.elapsed_time(e) / reps


def main(argv):
    if argv[0] == "train":
        B = int(argv[1])
        reps = int(argv[2]) if len(argv) > 2 else 3
        print(f"surrogate train step B={B} c=32 256x256: {surrogate_train(B, reps):.3f} ms", flush=True)
        return
    if argv[0] == "surrogate":
        B = int(argv[1])
        reps = int(argv[2]) if len(argv) > 2 else 5
        ms, fps, tf = surrogate_forward(B, reps)
        print(f"surrogate forward B={B} c=32 256x256: {ms:.4f} ms, {fps:.0f} frames/s, {tf:.1f} TFLOP/s", flush=True)
        return
    if argv[0] == "hist":
        B, H = int(argv[1]), int(argv[2])
        reps = int(argv[3]) if len(argv) > 3 else 10
        ms, gbs = hist_match(B, H, reps)
        print(f"hist_match B={B} H={H}: {ms:.4f} ms, {gbs:.1f} GB/s", flush=True)
        return
    kind, B, H, Cin, Cout = argv[0], *map(int, argv[1:5])
    stride = int(argv[5]) if len(argv) > 5 else 1
    reps = int(argv[6]) if len(argv) > 6 else 10
    ms, tf = conv3x3(kind, B, H, Cin, Cout, stride, reps)
    print(f"conv3x3 {kind} B={B} H={H} {Cin}->{Cout} stride {stride}: {ms:.4f} ms, {tf:.1f} TFLOP/s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
