"""Oracle of the learned surrogate (O3): plain PyTorch CPU float64.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg).

The learning-based simulator of SonoGym (Sec. 4; App. B.2 "Learning-based
approach") is a pix2pix U-Net from CT slices to ultrasound images, trained
with an L1 term (weight 1).  The surrogate here is the same kind of
network, an encoder-decoder with skip connections, mapping the label/HU
slice on the output grid to the physics frame.  The paper's figure of the
architecture is not in the text, so the layer list below is our reading:

    levels l = 0..3 with c * 2^l channels (c = base channels)
    encoder  level 0: conv3x3(8 -> c), conv3x3(c -> c)              -> e0
             level l: conv3x3 stride 2 (c_{l-1} -> c_l), conv3x3 x2 -> e_l
    decoder  level l = 2..0: convT2x2(c_{l+1} -> c_l), concat [up, e_l],
             conv3x3(2 c_l -> c_l), conv3x3(c_l -> c_l)
    head     1x1 conv (c -> 1), sigmoid
    every conv and convT is followed by ReLU (the head by the sigmoid)

Loss per frame (the pix2pix L1 term, plus a structural-similarity
term): L1 + (1 - SSIM), SSIM of Wang, Bovik, Sheikh,
Simoncelli 2004 (11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2,
C2 = 0.03^2, dynamic range 1, mean over the valid region).  Batch loss =
mean over frames.  Optimiser: Adam (Kingma & Ba 2015).

Tensor layouts follow the C ABI: activations NHWC; conv3x3 weights
[Cout][3][3][Cin]; convT2x2 weights [(dy*2+dx)*Cout + co][Cin]; head
weights [C]; the flat parameter vector lists, per layer in the order
above, the weights then the bias.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

DT = torch.float64
IN_CH = 8          # input channels (2 used: label / 4, clamp(HU / 1000, -1, 3); 6 zero)
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def layer_specs(c: int, levels: int = 4):
    """(name, kind, cin, cout, stride) in parameter order."""
    ch = [c * (2 ** l) for l in range(levels)]
    L = [("enc0a", "conv", IN_CH, ch[0], 1), ("enc0b", "conv", ch[0], ch[0], 1)]
    for l in range(1, levels):
        L += [(f"down{l}", "conv", ch[l - 1], ch[l], 2), (f"enc{l}a", "conv", ch[l], ch[l], 1),
              (f"enc{l}b", "conv", ch[l], ch[l], 1)]
    for l in range(levels - 2, -1, -1):
        L += [(f"up{l}", "convT", ch[l + 1], ch[l], 2), (f"dec{l}a", "conv", 2 * ch[l], ch[l], 1),
              (f"dec{l}b", "conv", ch[l], ch[l], 1)]
    L += [("head", "head", ch[0], 1, 1)]
    return L


def param_shapes(c: int, levels: int = 4):
    out = []
    for name, kind, cin, cout, s in layer_specs(c, levels):
        if kind == "conv":
            out += [(name + ".w", (cout, 3, 3, cin)), (name + ".b", (cout,))]
        elif kind == "convT":
            out += [(name + ".w", (4 * cout, cin)), (name + ".b", (cout,))]
        else:
            out += [(name + ".w", (cin,)), (name + ".b", (1,))]
    return out


def n_params(c: int, levels: int = 4) -> int:
    return sum(math.prod(s) for _, s in param_shapes(c, levels))


def unflatten(flat, c: int, levels: int = 4):
    flat = torch.as_tensor(flat, dtype=DT)
    P, o = {}, 0
    for name, shp in param_shapes(c, levels):
        n = math.prod(shp)
        P[name] = flat[o:o + n].reshape(shp)
        o += n
    assert o == flat.numel()
    return P


def conv3x3(x, w, b, stride, relu=True):
    """x [B][H][W][Cin], w [Cout][3][3][Cin]; zero padding 1."""
    y = F.conv2d(x.permute(0, 3, 1, 2), w.permute(0, 3, 1, 2), b, stride=stride, padding=1)
    y = y.permute(0, 2, 3, 1)
    return torch.relu(y) if relu else y


def convT2x2(x, w4, b, relu=True):
    """out[b, 2y+dy, 2x+dx, co] = sum_ci x[b, y, x, ci] w4[(2 dy + dx) Cout + co][ci] + bias[co]."""
    cout = w4.shape[0] // 4
    cin = w4.shape[1]
    wt = w4.reshape(2, 2, cout, cin).permute(3, 2, 0, 1)      # [Cin][Cout][dy][dx]
    y = F.conv_transpose2d(x.permute(0, 3, 1, 2), wt, b, stride=2).permute(0, 2, 3, 1)
    return torch.relu(y) if relu else y


def bf16_round(t):
    """round to the nearest bfloat16 (ties to even), back to float64"""
    return t.to(torch.bfloat16).to(DT)


def forward(P, x, c: int, levels: int = 4, keep=None, act=None):
    """x [B][H][W][8] -> frame [B][H][W] in (0, 1).

    act, if given, is applied to the output of every conv and convT (after
    its ReLU): the surrogate's stated precision keeps activations in BF16
    between layers (BF16 weights / activations, FP32 accumulation), which
    ``act=bf16_round`` restates; the default keeps float64 throughout."""
    A = act if act is not None else (lambda t: t)
    h = A(conv3x3(x, P["enc0a.w"], P["enc0a.b"], 1))
    skips = [A(conv3x3(h, P["enc0b.w"], P["enc0b.b"], 1))]
    h = skips[0]
    for l in range(1, levels):
        h = A(conv3x3(h, P[f"down{l}.w"], P[f"down{l}.b"], 2))
        h = A(conv3x3(h, P[f"enc{l}a.w"], P[f"enc{l}a.b"], 1))
        h = A(conv3x3(h, P[f"enc{l}b.w"], P[f"enc{l}b.b"], 1))
        skips.append(h)
    if keep is not None:
        keep["bottleneck"] = skips[-1]
    h = skips[-1]
    for l in range(levels - 2, -1, -1):
        u = A(convT2x2(h, P[f"up{l}.w"], P[f"up{l}.b"]))
        h = torch.cat([u, skips[l]], dim=-1)
        h = A(conv3x3(h, P[f"dec{l}a.w"], P[f"dec{l}a.b"], 1))
        h = A(conv3x3(h, P[f"dec{l}b.w"], P[f"dec{l}b.b"], 1))
        if keep is not None:
            keep[f"dec{l}"] = h
    z = (h * P["head.w"]).sum(-1) + P["head.b"]
    if keep is not None:
        keep["z"] = z
    return torch.sigmoid(z)


def gaussian_window(size=11, sigma=1.5):
    k = torch.arange(size, dtype=DT) - (size - 1) / 2
    g = torch.exp(-k * k / (2 * sigma * sigma))
    g = g / g.sum()
    return torch.outer(g, g)


def ssim_map(x, y, size=11, sigma=1.5):
    """x, y [B][H][W]; valid-region SSIM map [B][H-size+1][W-size+1]."""
    w = gaussian_window(size, sigma)[None, None]
    f = lambda t: F.conv2d(t[:, None], w)[:, 0]
    mx, my = f(x), f(y)
    sxx = f(x * x) - mx * mx
    syy = f(y * y) - my * my
    sxy = f(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def frame_losses(pred, target):
    """per-frame (L1, SSIM)"""
    l1 = (pred - target).abs().mean(dim=(1, 2))
    ss = ssim_map(pred, target).mean(dim=(1, 2))
    return l1, ss


def loss(pred, target):
    l1, ss = frame_losses(pred, target)
    return (l1 + (1.0 - ss)).mean()


def loss_and_grads(flat, x, target, c: int, levels: int = 4):
    """(loss, d loss / d flat params) by reverse-mode differentiation."""
    p = torch.as_tensor(flat, dtype=DT).clone().requires_grad_(True)
    P = unflatten(p, c, levels)
    out = forward(P, torch.as_tensor(x, dtype=DT), c, levels)
    L = loss(out, torch.as_tensor(target, dtype=DT))
    L.backward()
    return float(L.detach()), p.grad.detach().clone(), out.detach()


def adam_step(p, g, m, v, t, lr=2e-4, b1=0.9, b2=0.999, eps=1e-8):
    """one Adam update (step count t >= 1); returns new (p, m, v)"""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (torch.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- error gate
# The physics render judges the surrogate (the learned and the model-based
# simulators of App. B.2 side by side): a linear head on the network's
# bottleneck features predicts each frame's L1 gap to physics, and frames
# predicted over a threshold are re-rendered by physics.  READING (the
# paper has no gate): features = the channel means of the deepest encoder
# activation; the head is fitted by ridge regression with an unpenalised
# intercept.


def features(bottleneck):
    """[B][h][w][C] deepest activation -> [B][C] channel means"""
    return bottleneck.mean(dim=(1, 2))


def fit_error_head(feat, target, ridge):
    """argmin_(w, w0) sum_i (w . f_i + w0 - t_i)^2 + ridge |w|^2, by its
    normal equations [X^T X + diag(ridge, .., ridge, 0)] (w, w0) = X^T t with
    X = [f, 1], solved by a library linear solve in float64.  Returns the
    F + 1 coefficients (w, w0)."""
    import numpy as np
    f = np.asarray(feat, np.float64)
    t = np.asarray(target, np.float64)
    X = np.concatenate([f, np.ones((len(f), 1))], axis=1)
    A = X.T @ X
    A[np.arange(f.shape[1]), np.arange(f.shape[1])] += ridge
    return np.linalg.solve(A, X.T @ t)


def predict_error(coef, feat):
    """w . f + w0 per frame"""
    import numpy as np
    f = np.asarray(feat, np.float64)
    return f @ coef[:-1] + coef[-1]


# ------------------------------------------------------------- GAN term
# App. B.2 (learning-based approach) trains its pix2pix network with an L1
# term and a GAN term, weights 1 and 0.01.  READING (the discriminator is
# not described; pix2pix's is a conditional patch classifier): the
# discriminator sees the input slice and a frame, as 16 channels (the 8
# input channels, the frame, 7 zeros), through three 3x3 stride-2
# convolutions with ReLU (16 -> cd -> 2 cd -> 2 cd channels; ReLU where
# pix2pix has a leaky one, the activation the operators provide) and a 1x1
# head to one logit per patch of 8 x 8 pixels.  Losses, with BCE on logits
# averaged over every patch of every frame:
#   generator:     L1 + (1 - SSIM) + gan_weight * BCE(D(x, G(x)), 1)
#   discriminator: (BCE(D(x, y), 1) + BCE(D(x, G(x)), 0)) / 2
GAN_WEIGHT = 0.01
D_IN = 16


def disc_layer_specs(cd: int):
    return [("d1", "conv", D_IN, cd, 2), ("d2", "conv", cd, 2 * cd, 2), ("d3", "conv", 2 * cd, 2 * cd, 2),
            ("dhead", "head", 2 * cd, 1, 1)]


def disc_param_shapes(cd: int):
    out = []
    for name, kind, cin, cout, s in disc_layer_specs(cd):
        if kind == "conv":
            out += [(name + ".w", (cout, 3, 3, cin)), (name + ".b", (cout,))]
        else:
            out += [(name + ".w", (cin,)), (name + ".b", (1,))]
    return out


def disc_n_params(cd: int) -> int:
    return sum(math.prod(s) for _, s in disc_param_shapes(cd))


def disc_unflatten(flat, cd: int):
    flat = torch.as_tensor(flat, dtype=DT)
    P, o = {}, 0
    for name, shp in disc_param_shapes(cd):
        n = math.prod(shp)
        P[name] = flat[o:o + n].reshape(shp)
        o += n
    assert o == flat.numel()
    return P


def disc_input(x, y):
    """[B][H][W][16]: the 8 input channels, the frame, 7 zeros"""
    B, H, W, _ = x.shape
    z = torch.zeros((B, H, W, D_IN - IN_CH - 1), dtype=x.dtype)
    return torch.cat([x[..., :IN_CH], y[..., None], z], dim=-1)


def disc_forward(Pd, x, y, act=None):
    """patch logits [B][H/8][W/8] of the discriminator on (slice x, frame y)"""
    A = act if act is not None else (lambda t: t)
    h = A(disc_input(x, y))
    for name in ("d1", "d2", "d3"):
        h = A(conv3x3(h, Pd[name + ".w"], Pd[name + ".b"], 2))
    return (h * Pd["dhead.w"]).sum(-1) + Pd["dhead.b"]


def bce_logits(z, t):
    """mean over every element of the binary cross-entropy of logits z
    against target t in {0, 1}: log(1 + e^z) - t z"""
    return (F.softplus(z) - t * z).mean()


def gan_generator_loss(P, Pd, x, target, c: int, cd: int, gan_weight=GAN_WEIGHT):
    pred = forward(P, x, c)
    return loss(pred, target) + gan_weight * bce_logits(disc_forward(Pd, x, pred), 1.0), pred


def gan_generator_grads(flat, dflat, x, target, c: int, cd: int, gan_weight=GAN_WEIGHT):
    """(loss, d loss / d generator params) of the generator's combined loss,
    the discriminator held fixed"""
    p = torch.as_tensor(flat, dtype=DT).clone().requires_grad_(True)
    Pd = disc_unflatten(torch.as_tensor(dflat, dtype=DT), cd)
    L, _ = gan_generator_loss(unflatten(p, c), Pd, torch.as_tensor(x, dtype=DT), torch.as_tensor(target, dtype=DT),
                              c, cd, gan_weight)
    L.backward()
    return float(L.detach()), p.grad.detach().clone()


def disc_loss_and_grads(dflat, x, real, fake, cd: int):
    """(loss, d loss / d discriminator params) of
    (BCE(D(x, real), 1) + BCE(D(x, fake), 0)) / 2"""
    q = torch.as_tensor(dflat, dtype=DT).clone().requires_grad_(True)
    Pd = disc_unflatten(q, cd)
    x = torch.as_tensor(x, dtype=DT)
    L = 0.5 * (bce_logits(disc_forward(Pd, x, torch.as_tensor(real, dtype=DT)), 1.0) +
               bce_logits(disc_forward(Pd, x, torch.as_tensor(fake, dtype=DT)), 0.0))
    L.backward()
    return float(L.detach()), q.grad.detach().clone()
