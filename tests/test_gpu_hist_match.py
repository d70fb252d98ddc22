"""CT histogram matching on the GPU (Sec. 3: the learned simulator's input
CT slices are matched to a reference intensity histogram) against the
oracle: the standalone operation bit for bit (integer decisions, FP32
binning and bin centres), and the matched HU channel of the surrogate input
against the oracle's own slices."""
import numpy as np
import pytest

from oracle import hist_match as hm
from paper_2507_01152_gb300 import scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def sim():
    from simhelp import gpu_sim
    wl = scene.workload_c2(4)
    s = gpu_sim(wl)
    yield wl, s
    s.close()


def _images(rng, B, n):
    out = np.empty((B, n), np.float32)
    for b in range(B):
        c = rng.integers(0, 4, n)
        v = np.where(c == 0, rng.normal(40, 30, n), np.where(c == 1, rng.normal(-90, 25, n),
                     np.where(c == 2, rng.normal(900 + 50 * b, 300, n), rng.uniform(-1100, 3200, n))))
        out[b] = v
    out[0, :5] = [-5000.0, 5000.0, -1024.0, 3071.999, 0.0]   # below, above and on the bin range's edges
    return out


@pytest.mark.parametrize("n", [65536 + 37, 65536 + 36])     # scalar and four-pixel vector paths
@pytest.mark.parametrize("nb,h0,w", [(4096, -1024.0, 1.0), (16384, -1024.0, 0.25), (3, -100.0, 70.0), (1, 0.0, 1.0)])
def test_standalone_matches_oracle_bitwise(sim, nb, h0, w, n):
    wl, s = sim
    rng = np.random.default_rng(nb)
    B = 5
    hu = _images(rng, B, n)
    mask = (rng.random((B, n)) < 0.8).astype(np.uint8)
    mask[3] = 0                                             # an image with no considered pixel
    ref = hm.reference_cumulative(rng.gamma(2.5, 150.0, 50000) - 500.0, h0, w, nb)
    s.set_hu_reference(ref, h0, w)
    d_hu, d_mask = torch.from_numpy(hu).cuda(), torch.from_numpy(mask).cuda()
    out = torch.full_like(d_hu, np.nan)
    s.hist_match(d_hu, d_mask, out)
    got = out.cpu().numpy()
    for b in range(B):
        want = hm.match(hu[b], mask[b].astype(bool), ref, h0, w)
        assert np.array_equal(got[b], want), (b, np.argwhere(got[b] != want)[:5])
    # no mask: every pixel; in place
    s.hist_match(d_hu, None, d_hu)
    got = d_hu.cpu().numpy()
    for b in range(B):
        assert np.array_equal(got[b], hm.match(hu[b], None, ref, h0, w))
    s.check()


def test_arguments(sim):
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_INVALID_ARG
    wl, s = sim
    x = torch.zeros((2, 10), device="cuda")
    s.set_hu_reference(None, 0, 1)
    with pytest.raises(UsError) as e:
        s.hist_match(x, None, x)                            # no reference
    assert e.value.status == US_ERR_INVALID_ARG
    for bad in (np.array([3, 2, 5]), np.array([0, 0, 0]), np.array([-1, 2, 3])):
        with pytest.raises(UsError) as e:
            s.set_hu_reference(bad, 0.0, 1.0)
        assert e.value.status == US_ERR_INVALID_ARG
    with pytest.raises(UsError):
        s.set_hu_reference(np.array([1, 2]), 0.0, 0.0)      # zero bin width


def test_sample_slices_carry_the_matched_hu(sim):
    """surrogate input with a reference set: labels and fan flags as
    without it; the HU channel of in-fan pixels is bf16(clamp(matched HU /
    1000)) of the oracle's own FP64 slice (cast to FP32) matched by the
    oracle; outside the fan the sampled HU.  FP32 and FP64 trilinear HU may
    fall in different bins within rounding of a bin edge: at most 0.1% of
    the pixels may differ, by at most one BF16 step of a neighbouring bin."""
    import oracle
    wl, s = sim
    spec, lab, hu = wl.volumes[0]
    pr = wl.probes[0]
    B = 4
    envs, poses = wl.envs[:B], wl.poses[:B]
    other = scene.make_volume(scene.VolumeSpec(96, 96, 96, 0.5, 3, 4321))[1]
    h0, w, nb = -1024.0, 1.0, 4096
    ref = hm.reference_cumulative(other[other > -1000], h0, w, nb)
    P = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    H, W = pr.out_h, pr.out_w
    plain = torch.zeros((B, H, W, 8), dtype=torch.int16, device="cuda")
    s.set_hu_reference(None, 0, 1)
    s.sample_slices(envs, P, plain)
    s.set_hu_reference(ref, h0, w)
    got = torch.zeros_like(plain)
    s.sample_slices(envs, P, got)
    s.set_hu_reference(None, 0, 1)
    torch.cuda.synchronize()
    g = got.view(torch.bfloat16).float().cpu().numpy()
    p0 = plain.view(torch.bfloat16).float().cpu().numpy()
    assert np.array_equal(g[..., [0, 2, 3, 4, 5, 6, 7]], p0[..., [0, 2, 3, 4, 5, 6, 7]])
    bad = total = 0
    for b in range(B):
        raw = oracle.sample_slice_raw(lab, hu, spec.voxel_mm, pr, poses[b])
        fan = raw[..., 2] > 0
        m = hm.match(raw[..., 1].astype(np.float32).ravel(), fan.ravel(), ref, h0, w).reshape(H, W)
        want = torch.from_numpy(np.clip(m * np.float32(1e-3), -1, 3).astype(np.float32)).to(torch.bfloat16).float().numpy()
        ch = g[b, ..., 1]
        assert np.array_equal(ch[~fan], p0[b, ..., 1][~fan])
        diff = ch[fan] != want[fan]
        bad += int(diff.sum())
        total += int(fan.sum())
        assert abs(float(np.mean(ch[fan])) - float(np.mean(want[fan]))) < 1e-3
        assert abs(float(np.mean(ch[fan])) - float(np.mean(p0[b, ..., 1][fan]))) > 1e-2   # matching moved it
    assert bad <= 1e-3 * total, (bad, total)
