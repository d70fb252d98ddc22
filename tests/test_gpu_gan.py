"""The GAN term of the learned simulator (App. B.2: L1 and GAN terms,
weights 1 and 0.01) on the GPU against the float64 oracle O3: the
generator's gradient of its combined loss (the discriminator held fixed),
the discriminator's gradient of its own loss, and its Adam update."""
import math

import numpy as np
import pytest

from oracle import surrogate_ref as S
from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C, CD, H, W, B = 16, 16, 32, 32, 2


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()


def _disc_init(cd, seed):
    """He-normal weights N(0, 2 / fan_in) (the head N(0, 1 / fan_in)), zero biases"""
    rng = np.random.default_rng(seed)
    out = []
    for name, shp in S.disc_param_shapes(cd):
        n = math.prod(shp)
        if name.endswith(".w"):
            fan = shp[1] * shp[2] * shp[3] if len(shp) == 4 else shp[0]
            out.append(rng.normal(0, math.sqrt((2.0 if len(shp) == 4 else 1.0) / fan), n))
        else:
            out.append(np.zeros(n))
    return np.concatenate(out).astype(np.float32)


def _rounded(flat, shapes):
    """what the GPU computes with: convolution weights in BF16, the rest FP32"""
    out, o = torch.tensor(flat, dtype=torch.float64), 0
    for name, shp in shapes:
        n = math.prod(shp)
        if name.endswith(".w") and len(shp) == 4:
            out[o:o + n] = out[o:o + n].float().to(torch.bfloat16).double()
        else:
            out[o:o + n] = out[o:o + n].float().double()
        o += n
    return out


def _inputs(seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.zeros((B, H, W, 8), dtype=torch.float64)
    x[..., 0] = torch.randint(0, 5, (B, H, W), generator=g) / 4.0
    x[..., 1] = torch.rand((B, H, W), generator=g) * 2 - 0.5
    x[..., 2] = (torch.rand((B, H, W), generator=g) > 0.3).double()
    x = x.to(torch.bfloat16).double()
    t = torch.sigmoid(torch.nn.functional.avg_pool2d(x[..., 1][:, None], 5, 1, 2)[:, 0] * 3 - 1)
    return x, t.float().double()


def _net(gan_weight, dinit):
    from paper_2507_01152_gb300.ussim import Surrogate
    off, size, fan = Surrogate.segments(C, H, W)
    init = scene.surrogate_init(size, fan, 5)
    net = Surrogate(C, H, W, B, init, lr=2e-4)
    if gan_weight is not None:
        net.gan_enable(CD, dinit, gan_weight=gan_weight, lr=1e-3)
    return net, init


def _per_layer(a, b, shapes, min_cos, max_rel):
    o = 0
    for name, shp in shapes:
        n = math.prod(shp)
        x, y = a[o:o + n], b[o:o + n]
        if y.norm() > 1e-9:
            cos = float(x @ y / (x.norm() * y.norm()))
            assert cos > min_cos, (name, cos)
            assert float((x - y).norm() / y.norm()) < max_rel, name
        o += n


def test_generator_gradient_with_the_gan_term_matches_oracle():
    """The generator's gradient of L1 + (1 - SSIM) + w BCE(D(x, G(x)), 1),
    and the GAN term's own share (with minus without it), against O3; w = 1
    makes the term large enough to check, then the paper's 0.01."""
    dinit = _disc_init(CD, 3)
    x, t = _inputs(1)
    xd, td = x.to(torch.bfloat16).cuda(), t.float().cuda()
    P = _rounded(_net(None, None)[1], S.param_shapes(C))
    Pd = _rounded(dinit, S.disc_param_shapes(CD))
    plain, _ = _net(None, None)
    loss = torch.zeros(1 + 2 * B, device="cuda")
    plain.train_step(xd, td, loss, update=False)
    plain.check()
    g_plain = torch.tensor(plain.grads(), dtype=torch.float64)
    _, o_plain, _ = S.loss_and_grads(P, x, t, C)
    for w in (1.0, 0.01):
        net, _ = _net(w, dinit)
        net.train_step(xd, td, loss, update=False)
        net.check()
        L = float(loss[0])
        g = torch.tensor(net.grads(), dtype=torch.float64)
        Lo, go = S.gan_generator_grads(P, Pd, x, t, C, CD, gan_weight=w)
        assert abs(L - Lo) < 2e-2 * abs(Lo), (w, L, Lo)
        # per layer as the plain loss's gradient test (cosine 0.98), less the
        # discriminator's own BF16 layers on the GAN term's path (three more
        # data gradients in BF16 before the generator's output): 0.97
        _per_layer(g, go, S.param_shapes(C), 0.97, 0.25)
        total = float(g @ go / (g.norm() * go.norm()))
        assert total > 0.995, (w, total)
        if w == 1.0:
            share, oshare = g - g_plain, go - o_plain
            cos = float(share @ oshare / (share.norm() * oshare.norm()))
            assert float(oshare.norm()) > 0.05 * float(o_plain.norm())       # the term matters at this weight
            assert cos > 0.95, cos
        net.close()
    plain.close()


def test_discriminator_gradient_and_update_match_oracle():
    """(BCE(D(x, real), 1) + BCE(D(x, fake), 0)) / 2 over the
    discriminator, the fake frames being the generator's last output, against
    O3 fed the same (BF16-rounded) frames; then one Adam step."""
    dinit = _disc_init(CD, 4)
    x, t = _inputs(2)
    xd, td = x.to(torch.bfloat16).cuda(), t.float().cuda()
    net, _ = _net(0.01, dinit)
    loss = torch.zeros(1 + 2 * B, device="cuda")
    fake = torch.zeros((B, H, W), device="cuda")
    net.train_step(xd, td, loss, update=False)
    net.forward(xd, fake)
    l3 = torch.zeros(3, device="cuda")
    net.gan_disc_step(xd, td, l3, update=False)
    net.check()
    p0, gd = net.gan_params_grads()
    Pd = _rounded(dinit, S.disc_param_shapes(CD))
    real = t.to(torch.bfloat16).double()
    fk = fake.double().cpu().to(torch.bfloat16).double()
    Lo, go = S.disc_loss_and_grads(Pd, x, real, fk, CD)
    l3h = l3.cpu().numpy()
    assert abs(float(l3h[0]) - Lo) < 1e-3 * abs(Lo) + 1e-5, (l3h, Lo)
    assert abs(float(l3h[0]) - 0.5 * float(l3h[1] + l3h[2])) < 1e-6
    g = torch.tensor(gd, dtype=torch.float64)
    # the data gradients between the discriminator's layers are BF16 (2^-8
    # relative each), two to three layers deep for the first layers' weights
    _per_layer(g, go, S.disc_param_shapes(CD), 0.99, 0.1)
    # one Adam step from zero moments
    net.gan_disc_step(xd, td, l3, update=True)
    net.check()
    p1, g1 = net.gan_params_grads()
    want, _, _ = S.adam_step(torch.tensor(p0, dtype=torch.float64), torch.tensor(g1, dtype=torch.float64),
                             torch.zeros(len(p0), dtype=torch.float64), torch.zeros(len(p0), dtype=torch.float64), 1,
                             lr=1e-3)
    assert torch.allclose(torch.tensor(p1, dtype=torch.float64), want, rtol=0, atol=2e-6)
    net.close()
