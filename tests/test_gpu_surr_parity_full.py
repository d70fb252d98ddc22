"""The surrogate's operators and network at the production sizes (base 32
channels, 256 x 256 frames, batch 2) against the float64 oracle O3,
element by element.

Bounds, per element, on BF16-exact inputs and weights (products exact in
FP32):
* BF16 outputs: |g - o| <= 2^-8 |o| + 1e-4 A + 1e-6, where 2^-8 covers the
  rounding of the result to BF16 (half an ulp: at most 2^-8 relative) and
  A = sum |x| |w| over the element's terms bounds the FP32 accumulation
  (the worst case over n terms is n 2^-24 A, 1.4e-4 A for the widest
  layer's 2304 terms; a random-sign sum stays near sqrt(n) 2^-24 A);
* FP32 weight gradients: |g - o| <= 1e-4 A + 1e-6 |o|, A = sum |x| |dy|.
A wrong tile, tap or channel moves elements by a sizeable fraction of
their own magnitude and fails these bounds.

The whole network: O3 with its activations rounded to BF16 after every
layer (the surrogate's stated precision) against the GPU forward, pixel by
pixel; only the accumulation differs, which can move a BF16 rounding of an
activation by one unit in a few elements.  The bar is twice the distance
between two oracle evaluations of the same precision, one accumulating in
FP64 and one in FP32.
"""
import math

import numpy as np
import pytest

from oracle import surrogate_ref as S
from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()
    torch.set_num_threads(max(1, min(16, torch.get_num_threads())))


def bf(t):
    return t.to(torch.bfloat16).double()


def dev(t):
    return t.to(torch.bfloat16).contiguous().cuda()


def call(name, *args):
    from paper_2507_01152_gb300.ussim import op
    op(name, *args)
    torch.cuda.synchronize()


def relu_input(g, shape):
    return bf(torch.relu(torch.randn(shape, generator=g, dtype=torch.float64)))


def within(got, ref, A, rel_out, rel_acc, floor, what):
    err = (got - ref).abs()
    bound = rel_out * ref.abs() + rel_acc * A + floor
    worst = float((err / bound).max())
    assert worst <= 1.0, f"{what}: worst error / bound = {worst:.3f} (max err {float(err.max()):.3e})"
    return worst


CONV_SHAPES = [
    # B, H, W, Cin, Cout, stride, input channel stride, input channel offset   (layer)
    (2, 256, 256, 8, 32, 1, 8, 0),          # enc0a
    (2, 256, 256, 32, 32, 1, 32, 0),        # enc0b, dec0b
    (2, 256, 256, 64, 32, 1, 64, 0),        # dec0a (the concatenated skip)
    (2, 256, 256, 32, 64, 2, 32, 0),        # down1
    (2, 128, 128, 64, 64, 1, 64, 0),        # enc1a/b, dec1b
    (2, 64, 64, 128, 128, 1, 128, 0),       # enc2a/b, dec2b
    (2, 64, 64, 128, 256, 2, 128, 0),       # down3
    (2, 32, 32, 256, 256, 1, 256, 0),       # enc3a/b (bottleneck)
    (2, 128, 128, 128, 64, 1, 128, 0),      # dec1a (the concatenated skip)
    (2, 64, 64, 256, 128, 1, 256, 0),       # dec2a (the concatenated skip)
    (2, 256, 256, 32, 64, 2, 64, 32),       # down1 reading the skip half of its concatenation buffer
    (2, 256, 256, 32, 32, 1, 64, 32),       # a 32-channel haloed box read out of a 64-channel buffer
    (1, 40, 20, 128, 128, 1, 128, 0),       # streamed weights, ragged tiles (40 = 16 + 16 + 8 rows, 20 = 8 + 8 + 4)
    (3, 24, 36, 128, 128, 1, 256, 128),     # streamed weights, ragged, the upper half of a 256-channel buffer
]


@pytest.mark.parametrize("B,H,W,Cin,Cout,stride,cs_in,co_in", CONV_SHAPES)
def test_conv3x3_elementwise_production_shapes(B, H, W, Cin, Cout, stride, cs_in, co_in):
    g = torch.Generator().manual_seed(7 * H + Cin + 3 * Cout + stride)
    xfull = relu_input(g, (B, H, W, cs_in))
    x = xfull[..., co_in:co_in + Cin]
    w = bf(torch.randn((Cout, 3, 3, Cin), generator=g, dtype=torch.float64) * (2.0 / (9 * Cin)) ** 0.5)
    bias = (torch.randn(Cout, generator=g, dtype=torch.float64) * 0.1).float().double()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    # forward
    y = torch.zeros((B, Ho, Wo, Cout), dtype=torch.bfloat16, device="cuda")
    call("us_conv3x3_fwd", dev(xfull), cs_in, co_in, dev(w), bias.float().cuda(), y, Cout, 0, B, H, W, Cin, Cout,
         stride, 1, err)
    ref = S.conv3x3(x, w, bias, stride, relu=True)
    A = S.conv3x3(x.abs(), w.abs(), bias.abs(), stride, relu=False)
    within(y.double().cpu(), ref, A, 2.0 ** -8, 1e-4, 1e-6, "forward")
    # data gradient (dx masked by x > 0) and weight gradient of sum(dy * conv(x))
    dy = bf(torch.randn((B, Ho, Wo, Cout), generator=g, dtype=torch.float64))
    xr = x.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    out = S.conv3x3(xr, wr, bias, stride, relu=False)
    gx, gw = torch.autograd.grad(out, (xr, wr), dy)
    xa = x.abs().requires_grad_(True)
    wa = w.abs().requires_grad_(True)
    outa = S.conv3x3(xa, wa, None, stride, relu=False)
    Ax, Aw = torch.autograd.grad(outa, (xa, wa), dy.abs())
    mask = (x > 0).double()
    if Cin % 16 == 0:
        wd = w.permute(3, 1, 2, 0).contiguous()          # [Cin][3][3][Cout]
        dx = torch.zeros((B, H, W, Cin), dtype=torch.bfloat16, device="cuda")
        call("us_conv3x3_dgrad", dev(dy), Cout, 0, dev(wd), dev(xfull), cs_in, co_in, dx, Cin, 0, 0, B, H, W,
             Cin, Cout, stride, err)
        within(dx.double().cpu(), gx * mask, Ax * mask, 2.0 ** -8, 1e-4, 1e-6, "data gradient")
    gwt = torch.zeros((9 * Cin, Cout), dtype=torch.float32, device="cuda")
    call("us_conv3x3_wgrad", dev(xfull), cs_in, co_in, dev(dy), Cout, 0, gwt, B, H, W, Cin, Cout, stride, err)
    to_t = lambda t: t.permute(1, 2, 3, 0).reshape(9 * Cin, Cout)
    within(gwt.double().cpu(), to_t(gw), to_t(Aw), 1e-6, 1e-4, 1e-9, "weight gradient")
    assert int(err.item()) == 0


@pytest.mark.parametrize("Cin,Cout", [(32, 32), (8, 32), (64, 64)])
def test_conv3x3_writes_a_channel_window_of_a_wider_buffer(Cin, Cout):
    """The forward into channels [Cout, 2 Cout) of a 2 Cout-channel buffer
    (the encoder's skip into its concatenation buffer): the window holds the
    convolution, the other channels keep their contents."""
    B, H, W = 2, 256, 256
    g = torch.Generator().manual_seed(31 + Cin + Cout)
    x = relu_input(g, (B, H, W, Cin))
    w = bf(torch.randn((Cout, 3, 3, Cin), generator=g, dtype=torch.float64) * (2.0 / (9 * Cin)) ** 0.5)
    bias = (torch.randn(Cout, generator=g, dtype=torch.float64) * 0.1).float().double()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.full((B, H, W, 2 * Cout), 7.0, dtype=torch.bfloat16, device="cuda")
    call("us_conv3x3_fwd", dev(x), Cin, 0, dev(w), bias.float().cuda(), y, 2 * Cout, Cout, B, H, W, Cin, Cout, 1, 1,
         err)
    ref = S.conv3x3(x, w, bias, 1, relu=True)
    A = S.conv3x3(x.abs(), w.abs(), bias.abs(), 1, relu=False)
    within(y[..., Cout:].double().cpu(), ref, A, 2.0 ** -8, 1e-4, 1e-6, "window")
    assert bool((y[..., :Cout] == 7.0).all())
    assert int(err.item()) == 0


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 128, 128, 64, 32), (2, 64, 64, 128, 64), (2, 32, 32, 256, 128)])
def test_convT2x2_elementwise_production_shapes(B, H, W, Cin, Cout):
    g = torch.Generator().manual_seed(11 * H + Cin + Cout)
    x = relu_input(g, (B, H, W, Cin))
    w4 = bf(torch.randn((4 * Cout, Cin), generator=g, dtype=torch.float64) * (1.0 / Cin) ** 0.5)
    bias = (torch.randn(Cout, generator=g, dtype=torch.float64) * 0.1).float().double()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    # forward into the upsampled half of the decoder's concatenation buffer
    y = torch.zeros((B, 2 * H, 2 * W, 2 * Cout), dtype=torch.bfloat16, device="cuda")
    call("us_convT2x2_fwd", dev(x), Cin, 0, dev(w4), bias.float().cuda(), y, 2 * Cout, 0, B, H, W, Cin, Cout, 1, err)
    ref = S.convT2x2(x, w4, bias, relu=True)
    A = S.convT2x2(x.abs(), w4.abs(), bias.abs(), relu=False)
    within(y.double().cpu()[..., :Cout], ref, A, 2.0 ** -8, 1e-4, 1e-6, "forward")
    assert torch.all(y.double().cpu()[..., Cout:] == 0)
    dy = bf(torch.randn((B, 2 * H, 2 * W, Cout), generator=g, dtype=torch.float64))
    xr = x.clone().requires_grad_(True)
    wr = w4.clone().requires_grad_(True)
    gx, gw = torch.autograd.grad(S.convT2x2(xr, wr, bias, relu=False), (xr, wr), dy)
    xa = x.abs().requires_grad_(True)
    wa = w4.abs().requires_grad_(True)
    Ax, Aw = torch.autograd.grad(S.convT2x2(xa, wa, torch.zeros(Cout, dtype=torch.float64), relu=False), (xa, wa),
                                 dy.abs())
    mask = (x > 0).double()
    dx = torch.zeros((B, H, W, Cin), dtype=torch.bfloat16, device="cuda")
    call("us_convT2x2_dgrad", dev(dy), Cout, 0, dev(w4.T.contiguous()), dev(x), Cin, 0, dx, Cin, 0, 0,
         B, H, W, Cin, Cout, err)
    within(dx.double().cpu(), gx * mask, Ax * mask, 2.0 ** -8, 1e-4, 1e-6, "data gradient")
    g4 = torch.zeros((4 * Cout, Cin), dtype=torch.float32, device="cuda")
    call("us_convT2x2_wgrad", dev(x), Cin, 0, dev(dy), Cout, 0, g4, B, H, W, Cin, Cout, err)
    within(g4.double().cpu(), gw, Aw, 1e-6, 1e-4, 1e-9, "weight gradient")
    assert int(err.item()) == 0


def _net(c, H, W, Bmax, seed):
    from paper_2507_01152_gb300.ussim import Surrogate
    off, size, fan = Surrogate.segments(c, H, W)
    init = scene.surrogate_init(size, fan, seed)
    return Surrogate(c, H, W, Bmax, init), init


def _oracle_params(flat, c):
    """what the GPU computes with: conv / convT weights rounded to BF16, the rest FP32"""
    out, o = torch.tensor(flat, dtype=torch.float64), 0
    for name, shp in S.param_shapes(c):
        n = math.prod(shp)
        if name.endswith(".w") and not name.startswith("head"):
            out[o:o + n] = out[o:o + n].float().to(torch.bfloat16).double()
        else:
            out[o:o + n] = out[o:o + n].float().double()
        o += n
    return out


def _slices(B, H, W, seed):
    """surrogate inputs shaped like the sampled slices: label / 4 in steps of
    0.25, a smooth HU field, an inside-fan flag"""
    g = torch.Generator().manual_seed(seed)
    x = torch.zeros((B, H, W, 8), dtype=torch.float64)
    lab = torch.nn.functional.avg_pool2d(torch.rand((B, 1, H, W), generator=g), 9, 1, 4)[:, 0]
    x[..., 0] = torch.floor(lab * 5).clamp(0, 4) / 4.0
    x[..., 1] = torch.nn.functional.avg_pool2d(torch.randn((B, 1, H, W), generator=g), 7, 1, 3)[:, 0] * 2
    yy, xx = torch.meshgrid(torch.arange(H), torch.arange(W), indexing="ij")
    x[..., 2] = ((xx - W / 2).abs() < (yy + 8) * 0.6).double()
    return bf(x)


def test_network_forward_per_pixel_at_production_size():
    """c = 32, 256 x 256, two frames: every output pixel of the GPU forward
    against O3's BF16-activation forward (FP64 accumulation), and the
    bottleneck features of the error head within BF16 rounding of O3's.

    The per-pixel bar comes from the oracle itself: the same BF16-activation
    network accumulated in FP32 instead of FP64 (another valid evaluation
    of the stated precision) moves some activations across a BF16 rounding
    boundary, and its distance to the FP64 evaluation measures how far such
    flips carry to the output.  The GPU must stay within twice that
    distance, pixel by pixel (max) and on average (mean)."""
    c, H, W, B = 32, 256, 256, 2
    net, init = _net(c, H, W, B, seed=21)
    x = _slices(B, H, W, 5)
    y = torch.zeros((B, H, W), device="cuda")
    net.forward(x.to(torch.bfloat16).cuda(), y)
    feat = torch.zeros((B, 8 * c), device="cuda")
    net.features(B, feat)
    net.check()
    P = S.unflatten(_oracle_params(init, c), c)
    keep = {}
    with torch.no_grad():
        ref = S.forward(P, x, c, keep=keep, act=S.bf16_round)
        P32 = {k: v.float() for k, v in P.items()}
        ref32 = S.forward(P32, x.float(), c, act=lambda t: t.to(torch.bfloat16).float()).double()
    spread = (ref32 - ref).abs()
    got = y.double().cpu()
    d = (got - ref).abs()
    assert 0.02 < float(ref.std()) and 0.05 < float(ref.mean()) < 0.95      # not saturated
    assert 0 < float(spread.max()) < 2e-2
    assert float(d.max()) <= 2 * float(spread.max()), (float(d.max()), float(spread.max()))
    assert float(d.mean()) <= 2 * float(spread.mean()), (float(d.mean()), float(spread.mean()))
    fo = S.features(keep["bottleneck"])
    fg = feat.double().cpu()
    assert torch.all((fg - fo).abs() <= 2.0 ** -8 * fo.abs() + 1e-5), float((fg - fo).abs().max())


def test_error_head_fit_and_prediction_match_oracle():
    """us_surr_fit_error_head against the oracle's ridge regression (normal
    equations by a library solve), through us_surr_predict_error on the
    features of a forward pass."""
    c, H, W, B = 16, 64, 64, 8
    net, init = _net(c, H, W, B, seed=4)
    x = _slices(B, H, W, 9)
    y = torch.zeros((B, H, W), device="cuda")
    net.forward(x.to(torch.bfloat16).cuda(), y)
    F = 8 * c
    feat = torch.zeros((B, F), device="cuda")
    net.features(B, feat)
    fg = feat.double().cpu().numpy()
    rng = np.random.default_rng(3)
    n = 400
    ftrain = (fg.mean(0) + rng.normal(0, 1, (n, F)) * (fg.std(0) + 1e-3)).astype(np.float32)
    wtrue = rng.normal(0, 0.01, F)
    target = (ftrain @ wtrue + 0.05 + rng.normal(0, 1e-3, n)).astype(np.float32)
    for ridge in (0.0, 1e-2, 1.0):
        net.fit_error_head(ftrain, target, ridge=ridge)
        pred = torch.zeros(B, device="cuda")
        net.predict_error(B, pred)
        net.check()
        coef = S.fit_error_head(ftrain, target, ridge)
        want = S.predict_error(coef, fg)
        scale = np.abs(fg) @ np.abs(coef[:-1]) + abs(coef[-1])
        got = pred.double().cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-5 * scale + 1e-7), (ridge, got, want)
