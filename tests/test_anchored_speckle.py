"""Volume-anchored, multi-scale scatter maps (App. B.2: N0, N1 fixed over
3-D space, with multi-scale versions): the oracle pinned to closed forms
(unit variance, the correlation two samples inherit from the scales they
share, exact anchoring under probe motion), then the GPU paths against it."""
import math

import numpy as np
import pytest

import oracle
from paper_2507_01152_gb300 import scene


def _amp2(levels):
    w = [2.0 ** -k for k in range(levels)]
    return [x / sum(w) for x in w]          # a_k^2


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_maps_are_unit_normal(levels):
    rng = np.random.default_rng(levels)
    pos = rng.uniform(-500, 500, (4000, 3)).astype(np.float32)   # distinct cells at every scale
    v = np.array([oracle.anchored_noise(p, levels, 0.25, 0, 77) for p in pos])
    n = len(v)
    for j in range(2):
        m, var = v[:, j].mean(), v[:, j].var()
        assert abs(m) < 5 / math.sqrt(n)
        assert abs(var - 1) < 5 * math.sqrt(2 / n)
    assert abs(np.corrcoef(v[:, 0], v[:, 1])[0, 1]) < 5 / math.sqrt(n)   # N0, N1 independent


@pytest.mark.parametrize("levels", [2, 3])
def test_correlation_is_the_weight_of_the_shared_scales(levels):
    """Two samples in the same cell of scales 1 .. L-1 but different finest
    cells share exactly those scales' terms: corr = sum_{k >= 1} a_k^2."""
    c = 0.25
    rng = np.random.default_rng(10 + levels)
    coarse = c * 2 ** (levels - 1)
    base = (rng.integers(-300, 300, (3000, 3)) * coarse).astype(np.float32)   # centres of coarsest cells
    # two points 0.6 c on either side of a coarsest-cell centre along x (the
    # same cell at every scale k >= 1, whose half-edge is >= c) and 0.1 c off
    # it along y and z: neighbouring finest cells along x, the same along y, z
    off = np.float32(0.1 * c)
    p = base + off
    q = base + off
    p[:, 0] = base[:, 0] - np.float32(0.6 * c)
    q[:, 0] = base[:, 0] + np.float32(0.6 * c)
    a = np.array([oracle.anchored_noise(x, levels, c, 0, 5)[0] for x in p])
    b = np.array([oracle.anchored_noise(x, levels, c, 0, 5)[0] for x in q])
    want = sum(_amp2(levels)[1:])
    got = np.corrcoef(a, b)[0, 1]
    assert abs(got - want) < 5 * (1 - want ** 2) / math.sqrt(len(a)), (got, want)


def _tissue():
    T = scene.Tissue
    # water (never scatters) and one tissue without attenuation that almost
    # always scatters, so S = E0 * T with E constant
    return [T(0.0, 1.48, 0.0, 0.0, float("-inf")), T(0.0, 1.6, 1.0, 0.5, 3.0)]


def _slab(nz=180, ny=12, nx=16):
    lab = np.ones((nz, ny, nx), np.uint8)
    hu = np.full((nz, ny, nx), 40, np.int16)
    return lab, hu


def _pose(t):
    return np.array([[1, 0, 0, t[0]], [0, 1, 0, t[1]], [0, 0, 1, t[2]]], np.float32)


ANCH = scene.Options(1, 1, 1, 1, speckle_anchor=1, speckle_levels=2, speckle_cell_mm=0.25)


def test_maps_move_with_the_tissue_not_the_probe():
    """A probe moved one sample spacing (= one finest cell, all values
    dyadic) along its beam sees the same scatter values one sample earlier;
    the beam-keyed maps do not."""
    lab, hu = _slab()
    pr = scene.linear_probe(8, 256, 64.0, 0.5)          # dr = 0.25 mm
    a = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, ANCH, _pose((4.0, 3.0, 2.0)), seed=9)
    b = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, ANCH, _pose((4.0, 3.0, 2.25)), seed=9)
    assert np.array_equal(a["S"][:, 1:], b["S"][:, :-1])
    assert np.mean(a["S"] > 0) > 0.9                      # the maps really scatter
    beam = scene.Options(1, 1, 1, 1)
    c = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, beam, _pose((4.0, 3.0, 2.0)), seed=9)
    d = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, beam, _pose((4.0, 3.0, 2.25)), seed=9)
    assert not np.array_equal(c["S"][:, 1:], d["S"][:, :-1])


def test_maps_are_fixed_in_time_and_keyed_by_volume():
    lab, hu = _slab()
    pr = scene.linear_probe(8, 256, 64.0, 0.5)
    P = _pose((4.0, 3.0, 2.0))
    a = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, ANCH, P, seed=9, step=0)
    b = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, ANCH, P, seed=9, step=7, env=3)
    c = oracle.render_frame(lab, hu, 0.5, _tissue(), pr, ANCH, P, seed=9, vol_id=1)
    assert np.array_equal(a["S"], b["S"])                 # no step or env in the key
    assert not np.array_equal(a["S"], c["S"])             # each volume has its own maps
    assert np.all(np.isfinite(a["n1"]))


# ---------------------------------------------------------------- GPU parity

@pytest.mark.gpu
def test_gpu_anchored_maps_match_oracle():
    """GPU paths against the oracle with the anchored two-scale maps: the
    pre-PSF image sample by sample (an identity PSF), except where the
    oracle's N1 lies within 1e-4 of the density threshold (the FP32 and FP64
    decisions may differ there; either is valid); and the batched paths
    (cluster kernel, two grids, persistent grid) bit-identical to the plain
    kernels."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from simhelp import gpu_sim, render_gpu
    spec = scene.c1_spec()
    lab, hu = scene.make_volume(spec)
    tiny = dict(psf_sigma_ax_mm=1e-6, psf_sigma_lat_mm=1e-6)
    probes = [scene.linear_probe(40, 200, 80.0, 0.5, **tiny), scene.curvilinear_probe(48, 160, 70.0, 60.0, 30.0,
                                                                                         64, 48, **tiny)]
    poses = scene.dorsal_poses(spec, 6, 31)
    envs = np.stack([np.zeros(6), np.arange(6) % 2], axis=1).astype(np.int32)
    opt = scene.Options(1, 1, 0, 1, speckle_anchor=1, speckle_levels=2, speckle_cell_mm=0.3)
    wl = scene.Workload("anch", [(spec, lab, hu)], probes, envs, poses, options=opt, seed=4242)
    sim = gpu_sim(wl)
    outs = {}
    shapes = ((8, 32, 0), (1, 16, 0), (1, 16, 1))          # cluster, two grids, persistent grid
    for shape in shapes:
        sim.set_tuning(shape[0], shape[1], 0, shape[2])
        outs[shape] = render_gpu(sim, envs, poses, wl.seed, 3, path=0)
    outs["plain"] = render_gpu(sim, envs, poses, wl.seed, 3, path=1)
    for k in ("envelope", "frame"):
        for b in range(6):
            for shape in shapes:
                assert np.array_equal(outs[shape][b][k], outs["plain"][b][k]), (shape, k, b)
    tab = scene.tissue_table()
    mu1 = np.array([t.mu1 for t in tab])
    flagged = 0
    for b in range(6):
        o = oracle.render_frame(lab, hu, spec.voxel_mm, tab, probes[envs[b][1]], opt, poses[b], env=b,
                                seed=wl.seed, step=3)
        g = outs["plain"][b]
        assert np.array_equal(g["label"], o["label"])
        near = np.abs(o["n1"] - mu1[o["label"]]) < 1e-4
        flagged += int(near.sum())
        err = np.abs(g["envelope"] - o["S"])[~near].max() / np.abs(o["S"]).max()
        assert err < 1e-4, (b, err)
    assert flagged < 20
