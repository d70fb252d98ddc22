"""Pins of the surrogate oracle (O3) against facts outside itself (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import surrogate_ref as S


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv3x3_matches_direct_loops(stride):
    r = _rng(stride)
    B, H, W, Ci, Co = 2, 7, 6, 3, 4
    x = r.normal(size=(B, H, W, Ci))
    w = r.normal(size=(Co, 3, 3, Ci))
    b = r.normal(size=Co)
    got = S.conv3x3(torch.tensor(x), torch.tensor(w), torch.tensor(b), stride, relu=False).numpy()
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    ref = np.zeros((B, Ho, Wo, Co))
    for n in range(B):
        for yo in range(Ho):
            for xo in range(Wo):
                for co in range(Co):
                    acc = b[co]
                    for ky in range(3):
                        for kx in range(3):
                            yi, xi = yo * stride - 1 + ky, xo * stride - 1 + kx
                            if 0 <= yi < H and 0 <= xi < W:
                                acc += np.dot(w[co, ky, kx], x[n, yi, xi])
                    ref[n, yo, xo, co] = acc
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_convT2x2_matches_direct_scatter():
    r = _rng(3)
    B, H, W, Ci, Co = 2, 3, 4, 5, 3
    x = r.normal(size=(B, H, W, Ci))
    w4 = r.normal(size=(4 * Co, Ci))
    b = r.normal(size=Co)
    got = S.convT2x2(torch.tensor(x), torch.tensor(w4), torch.tensor(b), relu=False).numpy()
    ref = np.zeros((B, 2 * H, 2 * W, Co)) + b
    for n in range(B):
        for y in range(H):
            for xx in range(W):
                for dy in range(2):
                    for dx in range(2):
                        for co in range(Co):
                            ref[n, 2 * y + dy, 2 * xx + dx, co] += np.dot(w4[(2 * dy + dx) * Co + co], x[n, y, xx])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_ssim_identity_and_constant_images():
    r = _rng(4)
    x = torch.tensor(r.uniform(size=(2, 20, 24)))
    assert torch.allclose(S.ssim_map(x, x), torch.ones(1, dtype=S.DT))
    a, b = 0.3, 0.7
    xa, xb = torch.full((1, 16, 16), a, dtype=S.DT), torch.full((1, 16, 16), b, dtype=S.DT)
    want = (2 * a * b + S.SSIM_C1) / (a * a + b * b + S.SSIM_C1)     # sigmas vanish
    assert torch.allclose(S.ssim_map(xa, xb), torch.tensor(want, dtype=S.DT))


def test_ssim_map_matches_direct_window():
    r = _rng(5)
    x, y = r.uniform(size=(1, 17, 19)), r.uniform(size=(1, 17, 19))
    m = S.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()
    k = np.arange(11) - 5.0
    g1 = np.exp(-k * k / (2 * 1.5 ** 2))
    g = np.outer(g1, g1)
    g /= g.sum()
    for (i, j) in [(0, 0), (3, 5), (6, 8)]:
        px, py = x[0, i:i + 11, j:j + 11], y[0, i:i + 11, j:j + 11]
        mx, my = (g * px).sum(), (g * py).sum()
        vx = (g * (px - mx) ** 2).sum()
        vy = (g * (py - my) ** 2).sum()
        cxy = (g * (px - mx) * (py - my)).sum()
        want = ((2 * mx * my + 1e-4) * (2 * cxy + 9e-4)) / ((mx * mx + my * my + 1e-4) * (vx + vy + 9e-4))
        assert abs(m[0, i, j] - want) < 1e-12


def test_parameter_count_by_hand():
    c = 32
    conv = lambda ci, co: co * 9 * ci + co
    convT = lambda ci, co: 4 * co * ci + co
    want = (conv(8, 32) + conv(32, 32)
            + conv(32, 64) + 2 * conv(64, 64) + conv(64, 128) + 2 * conv(128, 128) + conv(128, 256) + 2 * conv(256, 256)
            + convT(256, 128) + conv(256, 128) + conv(128, 128)
            + convT(128, 64) + conv(128, 64) + conv(64, 64)
            + convT(64, 32) + conv(64, 32) + conv(32, 32) + 33)
    assert S.n_params(c) == want


def test_loss_gradient_matches_finite_differences():
    c, H = 2, 16
    r = _rng(6)
    shapes = S.param_shapes(c)
    flat = np.concatenate([r.normal(0, 0.4, size=math.prod(s)) for _, s in shapes])
    x = np.zeros((2, H, H, 8))
    x[..., :2] = r.uniform(0, 1, size=(2, H, H, 2))
    t = r.uniform(0.1, 0.9, size=(2, H, H))
    L, g, _ = S.loss_and_grads(flat, x, t, c)
    idx = r.choice(flat.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        Lp = S.loss_and_grads(fp, x, t, c)[0]
        Lm = S.loss_and_grads(fm, x, t, c)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - float(g[i])) <= 1e-6 + 1e-4 * abs(fd), (i, fd, float(g[i]))


def test_adam_matches_torch_optimizer():
    r = _rng(7)
    p0 = torch.tensor(r.normal(size=50))
    grads = [torch.tensor(r.normal(size=50)) for _ in range(5)]
    q = p0.clone().requires_grad_(True)
    opt = torch.optim.Adam([q], lr=2e-4, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.clone(), torch.zeros(50, dtype=S.DT), torch.zeros(50, dtype=S.DT)
    for t, g in enumerate(grads, 1):
        opt.zero_grad()
        q.grad = g.clone()
        opt.step()
        p, m, v = S.adam_step(p, g, m, v, t)
    assert torch.allclose(p, q.detach(), rtol=0, atol=1e-12)
    # first step moves every coordinate by about lr against the gradient's sign
    p1, _, _ = S.adam_step(p0, grads[0], torch.zeros(50, dtype=S.DT), torch.zeros(50, dtype=S.DT), 1)
    assert torch.allclose(p1 - p0, -2e-4 * torch.sign(grads[0]), atol=1e-9)


def test_bf16_round_is_round_to_nearest_even():
    """the BF16 activation rounding the parity tests restate: 8 significant
    bits, ties to even (values chosen by hand)"""
    v = torch.tensor([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 3.0 + 2 ** -7, -2.5, 0.0],
                     dtype=torch.float64)
    want = [1.0, 1.0, 1.0 + 2 ** -6, 1.0, 3.0, -2.5, 0.0]
    assert S.bf16_round(v).tolist() == want
    x = torch.randn(1000, dtype=torch.float64, generator=torch.Generator().manual_seed(2))
    r = S.bf16_round(x)
    assert torch.all((r - x).abs() <= 2.0 ** -8 * x.abs())          # half an ulp: at most 2^-8 relative


def test_bf16_forward_is_the_float64_forward_rounded_per_layer():
    """with act = identity the BF16 option changes nothing; with BF16
    rounding every activation the network output moves by no more than the
    per-layer rounding lets it"""
    c = 4
    P = S.unflatten(torch.randn(S.n_params(c), dtype=torch.float64, generator=torch.Generator().manual_seed(1)) * 0.3,
                    c)
    x = torch.rand((1, 16, 16, 8), dtype=torch.float64, generator=torch.Generator().manual_seed(2))
    a = S.forward(P, x, c)
    b = S.forward(P, x, c, act=lambda t: t)
    assert torch.equal(a, b)
    keep = {}
    q = S.forward(P, x, c, keep=keep, act=S.bf16_round)
    assert torch.equal(keep["bottleneck"], S.bf16_round(keep["bottleneck"]))
    assert 0 < float((q - a).abs().max()) < 0.05


def test_error_head_ridge_closed_forms():
    """The error head's ridge regression (unpenalised intercept):
    * ridge 0 on an exactly linear target recovers its coefficients;
    * one feature: w = sum (f - fbar)(t - tbar) / (sum (f - fbar)^2 + ridge),
      w0 = tbar - w fbar (the textbook closed form);
    * a huge ridge drives w to 0 and w0 to the mean target."""
    r = _rng(8)
    f = r.normal(size=(50, 3))
    coef = np.array([0.5, -2.0, 0.25, 1.5])
    t = f @ coef[:3] + coef[3]
    np.testing.assert_allclose(S.fit_error_head(f, t, 0.0), coef, rtol=1e-10, atol=1e-12)
    f1 = r.normal(size=(40, 1))
    t1 = r.normal(size=40)
    for lam in (0.0, 0.3, 7.0):
        fc, tc = f1[:, 0] - f1[:, 0].mean(), t1 - t1.mean()
        w = (fc @ tc) / (fc @ fc + lam)
        got = S.fit_error_head(f1, t1, lam)
        np.testing.assert_allclose(got, [w, t1.mean() - w * f1[:, 0].mean()], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(S.predict_error(got, f1), w * f1[:, 0] + got[1], rtol=1e-12)
    big = S.fit_error_head(f, t, 1e12)
    assert np.all(np.abs(big[:3]) < 1e-8) and abs(big[3] - t.mean()) < 1e-6


def test_bce_on_logits_closed_form_and_gradient():
    """BCE of logits, the textbook -[t log s(z) + (1 - t) log(1 - s(z))]
    with s the logistic function, and its gradient (s(z) - t) / n"""
    z = torch.tensor([-3.0, -0.5, 0.0, 0.7, 4.0], dtype=torch.float64, requires_grad=True)
    for t in (0.0, 1.0):
        s = 1.0 / (1.0 + torch.exp(-z.detach()))
        want = -(t * torch.log(s) + (1 - t) * torch.log(1 - s)).mean()
        L = S.bce_logits(z, t)
        assert abs(float(L.detach()) - float(want)) < 1e-14
        g, = torch.autograd.grad(L, z)
        assert torch.allclose(g, (s - t) / 5, rtol=1e-13, atol=1e-15)
    assert abs(float(S.bce_logits(torch.zeros(4, dtype=torch.float64), 1.0)) - math.log(2)) < 1e-15


def test_discriminator_shapes_input_and_parameter_count():
    cd = 8
    n = 9 * 16 * cd + cd + 9 * cd * 2 * cd + 2 * cd + 9 * 2 * cd * 2 * cd + 2 * cd + 2 * cd + 1
    assert S.disc_n_params(cd) == n
    g = torch.Generator().manual_seed(3)
    x = torch.rand((2, 32, 24, 8), dtype=torch.float64, generator=g)
    y = torch.rand((2, 32, 24), dtype=torch.float64, generator=g)
    d = S.disc_input(x, y)
    assert d.shape == (2, 32, 24, 16)
    assert torch.equal(d[..., :8], x) and torch.equal(d[..., 8], y) and torch.all(d[..., 9:] == 0)
    Pd = S.disc_unflatten(torch.randn(n, dtype=torch.float64, generator=g) * 0.2, cd)
    z = S.disc_forward(Pd, x, y)
    assert z.shape == (2, 4, 3)                       # one logit per 8 x 8 patch


def test_gan_generator_gradient_matches_finite_differences():
    """the combined generator loss L1 + (1 - SSIM) + 0.01 BCE(D(x, G(x)), 1)
    differentiated by autograd against central differences, on a tiny net"""
    c, cd = 4, 4
    g = torch.Generator().manual_seed(5)
    flat = torch.randn(S.n_params(c), dtype=torch.float64, generator=g) * 0.3
    dflat = torch.randn(S.disc_n_params(cd), dtype=torch.float64, generator=g) * 0.3
    x = torch.rand((1, 16, 16, 8), dtype=torch.float64, generator=g)
    t = torch.rand((1, 16, 16), dtype=torch.float64, generator=g)
    L, grad = S.gan_generator_grads(flat, dflat, x, t, c, cd, gan_weight=5.0)   # a large weight exposes the term
    idx = torch.randperm(flat.numel(), generator=g)[:6]
    for i in idx.tolist():
        e = torch.zeros_like(flat)
        e[i] = 1e-6
        Lp, _ = S.gan_generator_grads(flat + e, dflat, x, t, c, cd, gan_weight=5.0)
        Lm, _ = S.gan_generator_grads(flat - e, dflat, x, t, c, cd, gan_weight=5.0)
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - float(grad[i])) <= 1e-6 * max(1.0, abs(fd)), (i, fd, float(grad[i]))
    L0, g0 = S.gan_generator_grads(flat, dflat, x, t, c, cd, gan_weight=0.0)
    assert abs(L0 - S.loss_and_grads(flat, x, t, c)[0]) < 1e-12      # weight 0: the plain loss
