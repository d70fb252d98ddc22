"""The learned surrogate with its physics judge and fallback: what training
gains over the untrained network, the error head, and the gated mixed step
(frames predicted over the threshold are re-rendered by physics)."""
import numpy as np
import pytest

from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    from paper_2507_01152_gb300 import train as T
    build.build()
    probe = scene.curvilinear_probe(128, 256, 80.0, 60.0, 40.0, 128, 128)
    net, src, hist = T.train(160, batch=32, c=16, lr=2e-3, log_every=0, probe=probe, log=lambda *a: None)
    return T, net, src, hist


def test_training_gains_over_the_untrained_network(trained):
    T, net, src, hist = trained
    fresh = T.make_surrogate(16, src.B, 2e-3, 12345, src.probe.out_h, src.probe.out_w)
    l1_t, ss_t = T.evaluate(net, src, 3)
    l1_u, ss_u = T.evaluate(fresh, src, 3)
    assert l1_t < 0.5 * l1_u, (l1_t, l1_u)
    assert ss_t > ss_u + 0.2, (ss_t, ss_u)


def test_error_head_and_gated_fallback(trained):
    T, net, src, hist = trained
    feat, true_l1 = T.gate_samples(net, src, 8)
    net.fit_error_head(feat, true_l1, ridge=1e-2)
    # fresh held-out batch
    x, y = src.batch(T.HELD_OUT_SEED + 5000, 77)
    B = src.B
    surr = torch.zeros_like(y)
    net.forward(x, surr)
    pred_err = torch.zeros(B, device="cuda")
    net.predict_error(B, pred_err)
    met = torch.zeros(1 + 2 * B, device="cuda")
    net.metrics(surr, y, met)
    l1_true = met[1:1 + B].cpu().numpy()
    pe = pred_err.cpu().numpy()
    assert np.corrcoef(pe, l1_true)[0, 1] > 0.3            # the head ranks frames by their error
    thr = float(np.median(pe))
    gated = pe > thr
    s_, yy = surr.cpu().numpy(), y.cpu().numpy()
    old = src.sim.get_tuning()
    # cluster kernel, two-pass path and its persistent grid re-render the gated frames
    for shape in ((8, 32, 0), (1, 16, 0), (1, 16, 1)):
        src.sim.set_tuning(shape[0], shape[1], 1, shape[2])
        frames = torch.zeros_like(y)
        n_rendered = torch.zeros(1, dtype=torch.int32, device="cuda")
        T.mixed_step(src.sim, net, src.poses, src.seed, 77, x, frames, pred_err, thr, n_rendered, envs_c=src.envs_c)
        torch.cuda.synchronize()
        assert int(n_rendered.item()) == int(gated.sum())
        f = frames.cpu().numpy()
        for b in range(B):
            assert np.array_equal(f[b], yy[b] if gated[b] else s_[b]), (shape, b)
    src.sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"])
    net.metrics(frames, y, met)
    mixed_l1 = float(met[1:1 + B].mean())
    assert mixed_l1 <= float(l1_true.mean()) + 1e-7
    assert mixed_l1 < 0.75 * float(l1_true.mean())
