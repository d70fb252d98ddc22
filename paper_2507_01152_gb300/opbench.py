"""Timing of single surrogate operators on the GPU (CUDA events, after
warm-up): one 3x3 convolution pass of the tcgen05 implicit GEMM.

    python -m paper_2507_01152_gb300.opbench fwd|dgrad|wgrad B H Cin Cout [stride] [reps]

B images of H x H pixels (input grid), NHWC BF16 activations with random
values, Cin -> Cout channels.  Prints the time per call and the rate in
TFLOP/s (2 x 9 x Cin x Cout multiply-adds per output pixel)."""
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


def main(argv):
    kind, B, H, Cin, Cout = argv[0], *map(int, argv[1:5])
    stride = int(argv[5]) if len(argv) > 5 else 1
    reps = int(argv[6]) if len(argv) > 6 else 10
    ms, tf = conv3x3(kind, B, H, Cin, Cout, stride, reps)
    print(f"conv3x3 {kind} B={B} H={H} {Cin}->{Cout} stride {stride}: {ms:.4f} ms, {tf:.1f} TFLOP/s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
