"""Pins of the histogram-matching oracle (Sec. 3: the learned simulator's
input CT slices are matched to the intensity histogram of training CT
images): properties and closed forms that do not restate its code."""
import numpy as np

from oracle import hist_match as hm

H0, W, NB = -1024.0, 1.0, 4096


def _img(rng, n):
    # a CT-like mixture: soft tissue, fat, bone, air
    parts = [rng.normal(40, 30, n // 2), rng.normal(-90, 20, n // 4), rng.normal(900, 250, n // 8),
             rng.uniform(-1024, -900, n - n // 2 - n // 4 - n // 8)]
    return np.concatenate(parts).astype(np.float32)


def test_matching_to_its_own_histogram_gives_bin_centres():
    rng = np.random.default_rng(1)
    v = _img(rng, 5000)
    ref = hm.reference_cumulative(v, H0, W, NB)
    out = hm.match(v, None, ref, H0, W)
    want = (np.floor(v - np.float32(H0)) + 0.5 + H0).astype(np.float32)
    assert np.array_equal(out, want)


def test_translated_reference_translates_the_image():
    """integer-valued image, reference = the same values + 100 HU: every
    pixel moves by exactly 100 (bin m = k + 100), to its bin centre"""
    rng = np.random.default_rng(2)
    v = rng.integers(-300, 400, 3000).astype(np.float32)
    ref = hm.reference_cumulative(v + 100, H0, W, NB)
    out = hm.match(v, None, ref, H0, W)
    assert np.array_equal(out, v + np.float32(100.5))


def test_output_cumulative_counts_follow_the_reference():
    """after matching, at every reference bin m the image's cumulative
    share does not exceed the reference's, and falls short of it by less
    than one source bin: 0 <= R[m] n - S_out[m] N < max_bin_count * N"""
    rng = np.random.default_rng(3)
    v = _img(rng, 8000)
    refv = rng.gamma(3.0, 120.0, 20000) - 600.0      # a different CT-like distribution
    R = hm.reference_cumulative(refv, H0, W, NB)
    out = hm.match(v, None, R, H0, W)
    n, N = len(v), int(R[-1])
    S_out = np.cumsum(np.bincount(hm.bin_index(out, H0, W, NB), minlength=NB))
    kmax = np.bincount(hm.bin_index(v, H0, W, NB), minlength=NB).max()
    gap = R * n - S_out * N
    assert gap.min() >= 0
    assert gap.max() < kmax * N
    # and the matched image sits on reference bins' centres
    assert np.all(np.isin(hm.bin_index(out, H0, W, NB), np.nonzero(np.diff(np.concatenate([[0], R])))[0]))


def test_mapping_is_monotone_and_masked_pixels_are_untouched():
    rng = np.random.default_rng(4)
    v = _img(rng, 4000)
    mask = rng.random(4000) < 0.6
    R = hm.reference_cumulative(rng.normal(200, 300, 9000), H0, W, NB)
    out = hm.match(v, mask, R, H0, W)
    assert np.array_equal(out[~mask], v[~mask])
    o = np.argsort(v[mask], kind="stable")
    assert np.all(np.diff(out[mask][o]) >= 0)
    assert np.array_equal(hm.match(v, np.zeros(4000, bool), R, H0, W), v)


def test_brute_force_on_tiny_inputs():
    """direct loops over bins (no search, no vector cumulative sums)"""
    rng = np.random.default_rng(5)
    nb, h0, w = 12, -3.0, 0.5
    for trial in range(40):
        v = rng.uniform(-4.0, 4.0, int(rng.integers(1, 20))).astype(np.float32)
        refc = rng.integers(0, 4, nb)
        refc[int(rng.integers(0, nb))] += 1
        R = np.cumsum(refc)
        out = hm.match(v, None, R, h0, w)
        n, N = len(v), int(R[-1])
        for i in range(len(v)):
            k = min(max(int(np.floor((v[i] - np.float32(h0)) / np.float32(w))), 0), nb - 1)
            S_k = 0
            for j in range(len(v)):
                kj = min(max(int(np.floor((v[j] - np.float32(h0)) / np.float32(w))), 0), nb - 1)
                S_k += kj <= k
            m = 0
            while int(R[m]) * n < S_k * N:
                m += 1
            assert out[i] == np.float32(np.float32(m + 0.5) * np.float32(w) + np.float32(h0)), (trial, i)


def test_raw_slice_agrees_with_the_scaled_slice():
    """the unscaled HU of the raw slice, scaled and clamped, is the
    surrogate-input channel of the existing slice oracle"""
    import oracle
    from paper_2507_01152_gb300 import scene
    spec = scene.c1_spec()
    lab, hu = scene.make_volume(spec)
    pr = scene.curvilinear_probe(32, 64, 60.0, 60.0, 30.0, 48, 40)
    pose = scene.dorsal_poses(spec, 1, 5)[0]
    a = oracle.sample_slice(lab, hu, spec.voxel_mm, pr, pose)
    b = oracle.sample_slice_raw(lab, hu, spec.voxel_mm, pr, pose)
    assert np.array_equal(a[..., 0], b[..., 0] / 4.0)
    assert np.array_equal(a[..., 1], np.clip(b[..., 1] / 1000.0, -1.0, 3.0))
    assert np.array_equal(a[..., 2], b[..., 2])


def test_single_bin_references_are_closed_forms():
    """a reference with one non-empty bin m sends every considered pixel to
    that bin's centre; with one bin in all, to h0 + w/2"""
    rng = np.random.default_rng(6)
    v = _img(rng, 3000)
    for m in (0, 700, 1500, NB - 1):
        R = np.zeros(NB, np.int64)
        R[m:] = 5
        out = hm.match(v, None, R, H0, W)
        assert np.all(out == np.float32(np.float32(m + 0.5) * np.float32(W) + np.float32(H0))), m
    out = hm.match(v, None, np.array([7], np.int64), -20.0, 3.0)
    assert np.all(out == np.float32(-18.5))
