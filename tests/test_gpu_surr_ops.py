"""Surrogate operators (implicit-GEMM convolutions on tcgen05) against the
surrogate oracle on BF16-exact inputs: FP32 outputs within 1e-4
(rel. Frobenius), BF16 outputs within 4e-3."""
import numpy as np
import pytest

from oracle import surrogate_ref as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()


def bf(t):
    """round to bfloat16, keep as float64 CPU tensor"""
    return t.to(torch.bfloat16).double()


def dev(t):
    return t.to(torch.bfloat16).contiguous().cuda()


def rel(a, b):
    return float((a - b).norm() / max(b.norm(), 1e-30))


def call(name, *args):
    from paper_2507_01152_gb300.ussim import op
    op(name, *args)
    torch.cuda.synchronize()


def relu_input(g, shape):
    """a post-ReLU activation: about half zeros"""
    return bf(torch.relu(torch.randn(shape, generator=g, dtype=torch.float64)))


@pytest.mark.parametrize("B,H,W,Cin,Cout,stride,cs_in,co_in", [
    (2, 20, 20, 8, 32, 1, 8, 0), (2, 17, 23, 32, 64, 2, 64, 32), (2, 16, 16, 16, 16, 1, 32, 16), (1, 12, 12, 64, 256, 1, 64, 0),
    (3, 9, 10, 128, 128, 2, 256, 128),
    # shapes whose 128-pixel tiles are boxes of one image (tensor-copy loaders):
    # 64-channel taps (4 rows x 32), 32-channel taps on 256-wide rows read
    # from a channel slice, stride 2 with 64- and 32-channel taps, 8-channel taps
    (2, 32, 32, 64, 64, 1, 64, 0), (2, 8, 256, 32, 32, 1, 64, 32), (2, 32, 32, 64, 128, 2, 128, 64),
    (2, 64, 64, 32, 64, 2, 32, 0), (1, 16, 128, 8, 32, 1, 8, 0)])
def test_conv3x3_forward_dgrad_wgrad(B, H, W, Cin, Cout, stride, cs_in, co_in):
    g = torch.Generator().manual_seed(B * 1000 + H * 31 + Cin + Cout)
    xfull = relu_input(g, (B, H, W, cs_in))
    x = xfull[..., co_in:co_in + Cin]
    w = bf(torch.randn((Cout, 3, 3, Cin), generator=g, dtype=torch.float64) * (2.0 / (9 * Cin)) ** 0.5)
    bias = torch.randn(Cout, generator=g, dtype=torch.float64) * 0.1
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    # forward (into a channel slice of a wider output)
    y_cs, y_co = Cout + 32, 16
    y = torch.zeros((B, Ho, Wo, y_cs), dtype=torch.bfloat16, device="cuda")
    call("us_conv3x3_fwd", dev(xfull), cs_in, co_in, dev(w), bias.float().cuda(), y, y_cs, y_co, B, H, W, Cin, Cout,
         stride, 1, err)
    ref = S.conv3x3(x, w, bias, stride, relu=True)
    got = y.double().cpu()[..., y_co:y_co + Cout]
    assert rel(got, ref) < 4e-3
    assert torch.all(y.double().cpu()[..., :y_co] == 0) and torch.all(y.double().cpu()[..., y_co + Cout:] == 0)
    # gradients of sum(dy * conv(x)) (pre-activation), dx masked by x > 0
    dy = bf(torch.randn((B, Ho, Wo, Cout), generator=g, dtype=torch.float64))
    xr = x.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    out = S.conv3x3(xr, wr, bias, stride, relu=False)
    gx, gw = torch.autograd.grad(out, (xr, wr), dy)
    gx = gx * (x > 0)
    wd = w.permute(3, 1, 2, 0).contiguous()              # [Cin][3][3][Cout]
    prev = bf(torch.randn((B, H, W, cs_in), generator=g, dtype=torch.float64))
    if Cin % 16:
        # input gradients need Cin to fill whole 16-column tiles; the network's
        # only such layer reads the input slice, whose gradient is never needed
        from paper_2507_01152_gb300.ussim import UsError
        with pytest.raises(UsError):
            call("us_conv3x3_dgrad", dev(dy), Cout, 0, dev(wd), dev(xfull), cs_in, co_in, dev(prev), cs_in, co_in, 0,
                 B, H, W, Cin, Cout, stride, err)
    for acc in ((0, 1) if Cin % 16 == 0 else ()):
        dx = dev(prev)
        call("us_conv3x3_dgrad", dev(dy), Cout, 0, dev(wd), dev(xfull), cs_in, co_in, dx, cs_in, co_in, acc, B, H, W,
             Cin, Cout, stride, err)
        want = gx + (prev[..., co_in:co_in + Cin] if acc else 0)
        assert rel(dx.double().cpu()[..., co_in:co_in + Cin], want) < 4e-3
        assert torch.equal(dx.double().cpu()[..., :co_in], prev[..., :co_in])
    gwt = torch.full((9 * Cin, Cout), 0.5, dtype=torch.float32, device="cuda")
    call("us_conv3x3_wgrad", dev(xfull), cs_in, co_in, dev(dy), Cout, 0, gwt, B, H, W, Cin, Cout, stride, err)
    want = gw.permute(1, 2, 3, 0).reshape(9 * Cin, Cout) + 0.5
    assert rel(gwt.double().cpu(), want) < 1e-4
    assert int(err.item()) == 0


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 10, 12, 64, 32), (1, 8, 8, 256, 128), (2, 33, 5, 128, 64)])
def test_convT2x2_forward_dgrad_wgrad(B, H, W, Cin, Cout):
    g = torch.Generator().manual_seed(B * 100 + H + Cin + Cout)
    x = relu_input(g, (B, H, W, Cin))
    w4 = bf(torch.randn((4 * Cout, Cin), generator=g, dtype=torch.float64) * (1.0 / Cin) ** 0.5)
    bias = torch.randn(Cout, generator=g, dtype=torch.float64) * 0.1
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    y_cs, y_co = 2 * Cout, 0                      # the upsampled half of a concat buffer
    y = torch.zeros((B, 2 * H, 2 * W, y_cs), dtype=torch.bfloat16, device="cuda")
    call("us_convT2x2_fwd", dev(x), Cin, 0, dev(w4), bias.float().cuda(), y, y_cs, y_co, B, H, W, Cin, Cout, 1, err)
    ref = S.convT2x2(x, w4, bias, relu=True)
    assert rel(y.double().cpu()[..., :Cout], ref) < 4e-3
    dy = bf(torch.randn((B, 2 * H, 2 * W, Cout), generator=g, dtype=torch.float64))
    xr = x.clone().requires_grad_(True)
    wr = w4.clone().requires_grad_(True)
    out = S.convT2x2(xr, wr, bias, relu=False)
    gx, gw = torch.autograd.grad(out, (xr, wr), dy)
    gx = gx * (x > 0)
    dyfull = torch.zeros((B, 2 * H, 2 * W, 2 * Cout), dtype=torch.float64)
    dyfull[..., :Cout] = dy                        # read from a slice of a wider gradient
    dx = torch.zeros((B, H, W, Cin), dtype=torch.bfloat16, device="cuda")
    call("us_convT2x2_dgrad", dev(dyfull), 2 * Cout, 0, dev(w4.T.contiguous()), dev(x), Cin, 0, dx, Cin, 0, 0,
         B, H, W, Cin, Cout, err)
    assert rel(dx.double().cpu(), gx) < 4e-3
    g4 = torch.zeros((4 * Cout, Cin), dtype=torch.float32, device="cuda")
    call("us_convT2x2_wgrad", dev(x), Cin, 0, dev(dyfull), 2 * Cout, 0, g4, B, H, W, Cin, Cout, err)
    assert rel(g4.double().cpu(), gw) < 1e-4
    assert int(err.item()) == 0


def test_bad_arguments_are_rejected_before_launch():
    from paper_2507_01152_gb300.ussim import UsError, op
    t = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    b = torch.zeros(32, device="cuda")
    with pytest.raises(UsError):   # Cin not a multiple of 8
        op("us_conv3x3_fwd", t, 8, 0, t, b, t, 32, 0, 1, 2, 2, 6, 32, 1, 1, err)
    with pytest.raises(UsError):   # stride 3
        op("us_conv3x3_fwd", t, 8, 0, t, b, t, 32, 0, 1, 2, 2, 8, 32, 3, 1, err)
