"""Pins of the CPU oracle against facts outside itself (no GPU).

Each test ties the oracle to something it cannot satisfy by construction:
published known-answer vectors (Philox), a library routine (scipy's Gaussian
window), closed forms of the image model of App. B.2 (homogeneous decay,
a single planar interface), invariances (rigid motion of probe and volume
together, linearity in E0), and the pure-Python brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest
import scipy.signal.windows as sw

import oracle
from oracle import brute
from paper_2507_01152_gb300 import scene

GOLD = os.path.join(os.path.dirname(__file__), "golden")
NP_PER_DB = 1.0 / (20.0 * math.log10(math.e))      # 1 Np = 8.6859 dB


def f32(v):
    """descriptor values cross the C ABI as float32"""
    return float(np.float32(v))


def _kat():
    rows = []
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, want in _kat():
        assert list(oracle.philox4x32_10(ctr, key)) == want
        assert brute.philox(ctr, key) == want


def test_philox_two_implementations_agree():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64)
        assert list(oracle.philox4x32_10(ctr, key)) == brute.philox(ctr, key)


def _homog(shape, label):
    nz, ny, nx = shape
    return np.full(shape, label, np.uint8), np.zeros(shape, np.int16)


def _axis_pose(R_cols, t):
    R = np.stack([np.asarray(c, float) for c in R_cols], axis=1)
    return np.concatenate([R, np.asarray(t, float)[:, None]], axis=1).astype(np.float32)


def test_speckle_statistics():
    """With unit scatter statistics, no attenuation, no interfaces and no
    PSF the envelope is the noise itself: N0 must be standard normal and
    the density test must pass with probability Phi(mu1)."""
    mu1 = 0.3
    table = [scene.Tissue(0.0, 1.5, 0.0, 0.0, -math.inf),
             scene.Tissue(0.0, 1.5, 0.0, 1.0, math.inf),
             scene.Tissue(0.0, 1.5, 0.0, 1.0, mu1)]
    lab, hu = _homog((40, 40, 40), 1)
    probe = scene.linear_probe(64, 512, 30.0, 0.25, psf_sigma_ax_mm=0.0, psf_sigma_lat_mm=0.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (20.0, 20.0, 2.0))
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 0, 1, 1), pose,
                              env=1, seed=77, step=3)
    n0 = res["envelope"].ravel()
    n = n0.size
    assert abs(n0.mean()) < 5 / math.sqrt(n)
    assert abs(n0.var() - 1) < 5 * math.sqrt(2 / n)
    kurt = np.mean(n0 ** 4) / n0.var() ** 2
    assert abs(kurt - 3) < 5 * math.sqrt(24 / n)
    # even samples take the cosine branch, odd the sine: both standard normal and
    # uncorrelated within a pair
    ev, od = res["envelope"][:, 0::2].ravel(), res["envelope"][:, 1::2].ravel()
    assert abs(np.corrcoef(ev, od)[0, 1]) < 5 / math.sqrt(ev.size)
    lab[:] = 2
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 0, 1, 1), pose,
                              env=1, seed=77, step=3)
    frac = np.mean(res["envelope"] != 0.0)
    p = 0.5 * math.erfc(-mu1 / math.sqrt(2))
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_psf_taps_match_scipy_gaussian_window():
    for sigma, d in [(0.3, 80.0 / 512), (1.0, 80.0 * math.pi / 3 / 255), (0.6, 0.5), (1.0, 0.5)]:
        taps = oracle.psf_taps(sigma, d)
        K = len(taps) // 2
        assert K == math.ceil(3 * sigma / d)
        ref = sw.gaussian(2 * K + 1, std=sigma / d)
        np.testing.assert_allclose(taps, ref / ref.sum(), rtol=1e-13, atol=1e-16)
    # curvilinear 256 x 512 probe, 60 deg fan, r0 40 mm, depth 80 mm:
    # axial 0.3 mm -> 13 taps, lateral 1 mm at rho = 80 mm -> 21 taps
    assert len(oracle.psf_taps(0.3, 80.0 / 512)) == 13
    assert len(oracle.psf_taps(1.0, 80.0 * math.radians(60.0) / 255)) == 21


def test_homogeneous_medium_decays_exponentially():
    """One tissue, no speckle, no interfaces: E = E0 exp(-f alpha y), so
    consecutive interior envelope samples differ by the one-sample decay."""
    alpha_db = 1.1
    table = [scene.Tissue(0.0, 1.5, 0.0, 0.0, -math.inf), scene.Tissue(alpha_db, 1.6, 1.0, 0.0, 0.0)]
    lab, hu = _homog((96, 48, 48), 1)
    probe = scene.linear_probe(32, 256, 80.0, 0.5, f_mhz=5.0, e0=2.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (24.0, 24.0, 4.0))
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 1, 1, 0), pose)
    I = res["envelope"]
    dr = 80.0 / 256
    c = 5.0 * f32(alpha_db) * NP_PER_DB * (dr / 10.0)   # Np per sample
    Ka = len(oracle.psf_taps(0.3, dr)) // 2
    Kl = len(oracle.psf_taps(1.0, 0.5)) // 2
    inner = I[Kl:-Kl, Ka:-Ka - 1]
    ratio = np.log(I[Kl:-Kl, Ka:-Ka - 1]) - np.log(I[Kl:-Kl, Ka + 1:-Ka])
    np.testing.assert_allclose(ratio, c, rtol=1e-10)
    # laterally constant away from the edge lines
    np.testing.assert_allclose(inner, np.broadcast_to(inner[0:1], inner.shape), rtol=1e-12)
    # energy itself: E_s = E0 exp(-c s)
    s = np.arange(256)
    np.testing.assert_allclose(res["E"][5], 2.0 * np.exp(-c * s), rtol=1e-12)


def _partial_tap_sums(taps, n):
    """W[i] = the sum of the taps that land inside [0, n) around index i
    (zero padding at the borders)"""
    K = len(taps) // 2
    return np.array([sum(taps[k + K] for k in range(-K, K + 1) if 0 <= i + k < n) for i in range(n)])


@pytest.mark.parametrize("probe_kind", ["linear", "curvilinear"])
def test_homogeneous_backscatter_is_energy_times_blurred_scatter(probe_kind):
    """App. B.2 fixes the backscatter as B = E . (P (x) T): the scatter
    pattern is blurred, then scaled by the energy at the pixel itself.  In a
    homogeneous attenuating medium with speckle off, T = mu0 everywhere in the
    volume and there are no interfaces, so the whole envelope is the closed
    form I(l, s) = E(l, s) mu0 W_lat(l) W_ax(s), W the sums of the taps that
    fall inside the frame (1 in the interior): I = E mu0 exactly away from the
    borders.  Blurring E . T instead (P (x) (E T)) would give
    E_s mu0 sum_k w_k e^(-c k) in the interior, which differs by far more than
    the tolerance here."""
    alpha_db, mu0 = 1.1, 0.7
    table = [scene.Tissue(0.0, 1.5, 0.0, 0.0, -math.inf), scene.Tissue(alpha_db, 1.6, mu0, 0.0, 0.0)]
    lab, hu = _homog((160, 160, 160), 1)
    if probe_kind == "linear":
        probe = scene.linear_probe(32, 256, 80.0, 0.5, f_mhz=5.0, e0=2.0)
        pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (80.0, 80.0, 4.0))
        dlat = f32(0.5)
    else:
        probe = scene.curvilinear_probe(48, 200, 60.0, 50.0, 30.0, 64, 48, f_mhz=5.0, e0=2.0)
        pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (80.0, 80.0, 4.0))
        dlat = (f32(30.0) + 0.5 * f32(60.0)) * math.radians(f32(50.0)) / 47
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 1, 1, 0), pose)
    NL, NS = probe.n_lines, probe.n_samples
    dr = f32(probe.depth_mm) / NS
    assert np.all(res["label"] == 1)                            # every sample inside the tissue
    wax = oracle.psf_taps(f32(0.3), dr)
    wlat = oracle.psf_taps(f32(1.0), dlat)
    want = res["E"] * f32(mu0) * np.outer(_partial_tap_sums(wlat, NL), _partial_tap_sums(wax, NS))
    np.testing.assert_allclose(res["envelope"], want, rtol=1e-12)
    c = 5.0 * f32(alpha_db) * NP_PER_DB * (dr / 10.0)
    s = np.arange(NS)
    np.testing.assert_allclose(res["E"], np.broadcast_to(2.0 * np.exp(-c * s), (NL, NS)), rtol=1e-12)
    Ka, Kl = len(wax) // 2, len(wlat) // 2
    inner = (slice(Kl, NL - Kl), slice(Ka, NS - Ka))
    np.testing.assert_allclose(res["envelope"][inner], f32(mu0) * res["E"][inner], rtol=1e-12)
    # the other composition's interior value is distinguishable at this tolerance
    other = f32(mu0) * res["E"][inner] * sum(w * math.exp(-c * k) for k, w in zip(range(-Ka, Ka + 1), wax))
    assert np.min(np.abs(other / res["envelope"][inner] - 1)) > 1e-5


def test_backscatter_blurs_the_pattern_not_the_energy_brute_force():
    """The same composition in the pure-Python brute force (full 2-D sums),
    with an energy that varies across the PSF support (bone-like attenuation)
    and speckle on: I = P (x) R_imp + E (P (x) T) term by term."""
    table = [scene.Tissue(0.0, 1.48, 0.0, 0.0, -math.inf), scene.Tissue(20.0, 1.6, 0.8, 0.3, 0.8)]
    lab, hu = _homog((12, 12, 12), 1)
    probe = scene.linear_probe(5, 24, 6.0, 0.5, psf_sigma_ax_mm=0.5, psf_sigma_lat_mm=0.6)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (6.0, 6.0, 2.0))
    b = brute.render(lab, hu, 1.0, table, probe, scene.Options(1, 1, 1, 1), pose, env=2, seed=5, step=1)
    dr = f32(6.0) / 24
    wax = oracle.psf_taps(f32(0.5), dr)
    wlat = oracle.psf_taps(f32(0.6), f32(0.5))
    P2 = np.outer(wlat, wax)
    Ka, Kl = len(wax) // 2, len(wlat) // 2
    Tp = np.pad(b["T"], ((Kl, Kl), (Ka, Ka)))
    blurred = np.array([[np.sum(P2 * Tp[l:l + 2 * Kl + 1, s:s + 2 * Ka + 1]) for s in range(24)] for l in range(5)])
    np.testing.assert_allclose(b["envelope"], b["E"] * blurred, rtol=1e-12, atol=1e-300)
    o = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 1, 1, 1), pose, env=2, seed=5, step=1)
    np.testing.assert_allclose(o["envelope"], b["envelope"], rtol=1e-12)
    np.testing.assert_array_equal(o["T"], b["T"])


@pytest.mark.parametrize("mu0, want", [(1.0, 1.0), (10.0 ** -1.5, 0.5), (1e-3, 0.0), (0.0, 0.0), (-1.0, 0.0),
                                       (10.0 ** -0.75, 0.75), (1e-4, 0.0), (3.0, 1.0)])
def test_log_compression_closed_forms(mu0, want):
    """Log compression y = clamp((20 log10(I / E0) + DR) / DR, 0, 1),
    DR = 60 dB: with no attenuation, no interfaces, no speckle and no PSF the
    envelope is I = E0 mu0 everywhere, so I = E0 gives 1, I = E0 10^(-DR/20)
    gives 0, 30 dB below E0 gives 0.5, I <= 0 and anything below the range
    give 0, anything above E0 gives 1."""
    table = [scene.Tissue(0.0, 1.5, 0.0, 0.0, -math.inf), scene.Tissue(0.0, 1.6, mu0, 0.0, 0.0)]
    lab, hu = _homog((40, 40, 40), 1)
    probe = scene.linear_probe(8, 64, 20.0, 0.5, e0=3.0, psf_sigma_ax_mm=0.0, psf_sigma_lat_mm=0.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (20.0, 20.0, 4.0))
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 1, 1, 0), pose)
    np.testing.assert_allclose(res["envelope"], 3.0 * f32(mu0), rtol=1e-15)
    np.testing.assert_allclose(res["logimg"], want, atol=1e-6)   # mu0 crosses the ABI as float32
    np.testing.assert_allclose(res["frame"], res["logimg"].T, atol=0)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("tau", [0, 1])
def test_single_planar_interface(p, tau):
    """Two tissues meeting on a plane perpendicular to the beam, no
    scatter: the only echo is the interface, |E r|^p with
    r = (Z2 - Z1)/(Z2 + Z1), blurred by the axial PSF; below it the energy
    carries the transmission factor (1 - r^2) when enabled."""
    a1, a2, Z1, Z2 = 0.5, 1.1, 1.38, 1.70
    table = [scene.Tissue(0.0, 1.5, 0.0, 0.0, -math.inf), scene.Tissue(a1, Z1, 0.0, 0.0, 0.0),
             scene.Tissue(a2, Z2, 0.0, 0.0, 0.0)]
    shape = (96, 48, 48)
    lab, hu = _homog(shape, 1)
    kb = 40
    lab[kb:] = 2
    probe = scene.linear_probe(32, 256, 80.0, 0.5, f_mhz=5.0, e0=1.0)
    tz = 4.0 + 1.0 / 32
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (24.0 + 1 / 32, 24.0 + 1 / 32, tz))
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(p, tau, 1, 0), pose)
    dr = 80.0 / 256
    # interface sample: the last sample whose nearest voxel lies above plane kb
    s_star = max(s for s in range(256) if math.floor(s * dr + tz + 0.5) < kb)
    r = (f32(Z2) - f32(Z1)) / (f32(Z2) + f32(Z1))
    c1 = 5.0 * f32(a1) * NP_PER_DB * dr / 10.0
    c2 = 5.0 * f32(a2) * NP_PER_DB * dr / 10.0
    Ka = math.ceil(3 * f32(0.3) / dr)
    wax = sw.gaussian(2 * Ka + 1, std=f32(0.3) / dr)
    wax /= wax.sum()
    Kl = math.ceil(3 * 1.0 / 0.5)
    peak = math.exp(-c1 * s_star) * abs(r) ** p
    I = res["envelope"][Kl:-Kl]
    for k in range(-Ka, Ka + 1):
        np.testing.assert_allclose(I[:, s_star + k], wax[k + Ka] * peak, rtol=1e-10)
    assert np.all(I[:, :s_star - Ka] == 0) and np.all(I[:, s_star + Ka + 1:] == 0)
    E = res["E"][10]
    m = np.arange(256 - s_star - 1)
    want = np.exp(-c1 * (s_star + 1) - c2 * m) * ((1 - r * r) if tau else 1.0)
    np.testing.assert_allclose(E[s_star + 1:], want, rtol=1e-11)


@pytest.mark.parametrize("phi_deg", [5.0, 10.0, 20.0, 30.0, 40.0])
def test_tilted_interface_incidence(phi_deg):
    """A plane tilted by phi against the beam-normal: the incidence
    estimate from the label slice averages to tan(phi) over the lines."""
    table = [scene.Tissue(0.0, 1.5, 0.0, 0.0, -math.inf), scene.Tissue(0.5, 1.4, 0.0, 0.0, 0.0),
             scene.Tissue(0.5, 1.7, 0.0, 0.0, 0.0)]
    n = 160
    x = np.arange(n)
    # tissue 2 below z = 60 + tan(phi) * (x - 80)   (volume axes: x = i, beam = +k)
    zb = 60.0 + math.tan(math.radians(phi_deg)) * (x - 80.0)
    k = np.arange(n)[:, None, None]
    lab = np.where(k >= zb[None, None, :], 2, 1).astype(np.uint8)
    lab = np.broadcast_to(lab, (n, 8, n)).copy()
    hu = np.zeros_like(lab, np.int16)
    probe = scene.linear_probe(96, 512, 60.0, 0.5, psf_sigma_ax_mm=0.0, psf_sigma_lat_mm=0.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (80.0 + 1 / 32, 4.0, 30.0 + 1 / 32))
    res = oracle.render_frame(lab, hu, 1.0, table, probe, scene.Options(1, 0, 1, 0), pose)
    G = (res["label"][:, 1:] != res["label"][:, :-1])
    ct = res["cos_theta"][:, :-1][G]
    tan_est = np.sqrt(1.0 / ct ** 2 - 1.0)
    # the interface steps by tan(phi) * pitch / dr samples per line; the mean
    # estimate recovers tan(phi) (quantisation averages out over the lines)
    assert abs(tan_est[2:-2].mean() - math.tan(math.radians(phi_deg))) < 0.12 * math.tan(math.radians(phi_deg)) + 0.01


def _rigid_case():
    rng = np.random.default_rng(11)
    shape = (24, 20, 28)   # nz, ny, nx
    lab = np.repeat(rng.integers(0, 5, (shape[0], shape[1], shape[2] // 4)), 4, axis=2).astype(np.uint8)
    hu = rng.integers(-300, 900, shape).astype(np.int16)
    probe = scene.linear_probe(12, 40, 12.5, 0.5, psf_sigma_ax_mm=0.5, psf_sigma_lat_mm=0.7)
    # beam along +y, lines along +x; translations off the half-voxel ties
    pose = _axis_pose([(1, 0, 0), (0, 0, 1), (0, 1, 0)], (10.0 + 1 / 32, 3.0 + 1 / 32, 11.0 + 3 / 32))
    return lab, hu, probe, pose


def _apply(lab, hu, pose, Fm, c, perm_flip):
    """Volume transformed so that voxel q of the new grid equals voxel
    F^-1 (q - c) of the old one; pose composed with p -> F p + c."""
    lab2, hu2 = perm_flip(lab), perm_flip(hu)
    R, t = pose[:, :3].astype(float), pose[:, 3].astype(float)
    pose2 = np.concatenate([Fm @ R, (Fm @ t + c)[:, None]], axis=1).astype(np.float32)
    return lab2, hu2, pose2


def test_rigid_invariance():
    lab, hu, probe, pose = _rigid_case()
    nz, ny, nx = lab.shape
    opts = scene.Options(1, 1, 0, 1)
    table = scene.tissue_table()
    ref = oracle.render_frame(lab, hu, 1.0, table, probe, opts, pose, env=2, seed=9, step=1)
    cases = []
    # 180 deg about z: x -> nx-1-x, y -> ny-1-y
    Fz = np.diag([-1.0, -1.0, 1.0])
    cases.append((Fz, np.array([nx - 1, ny - 1, 0.0]), lambda a: a[:, ::-1, ::-1]))
    # 90 deg about z: (x, y) -> (ny-1-y, x); new array [k][x][ny-1-y]
    F90 = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    cases.append((F90, np.array([ny - 1, 0.0, 0.0]), lambda a: np.ascontiguousarray(a.transpose(0, 2, 1)[:, :, ::-1])))
    # integer translation by padding
    pad = ((3, 0), (2, 0), (5, 0))
    cases.append((np.eye(3), np.array([5.0, 2.0, 3.0]), lambda a: np.pad(a, pad)))
    for Fm, c, pf in cases:
        lab2, hu2, pose2 = _apply(lab, hu, pose, Fm, c, pf)
        got = oracle.render_frame(lab2, hu2, 1.0, table, probe, opts, pose2, env=2, seed=9, step=1)
        assert np.array_equal(got["label"], ref["label"])
        np.testing.assert_allclose(got["envelope"], ref["envelope"], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(got["frame"], ref["frame"], rtol=0, atol=1e-12)


def test_linear_in_e0():
    lab, hu, probe, pose = _rigid_case()
    table = scene.tissue_table()
    opts = scene.Options(1, 1, 0, 1)
    a = oracle.render_frame(lab, hu, 1.0, table, probe, opts, pose, seed=4)
    import dataclasses
    probe3 = dataclasses.replace(probe, e0=3.0)
    b = oracle.render_frame(lab, hu, 1.0, table, probe3, opts, pose, seed=4)
    np.testing.assert_allclose(b["envelope"], 3.0 * a["envelope"], rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(b["frame"], a["frame"], atol=1e-12)


def test_nearest_index_and_hu_at_voxel_centres():
    """Axis-aligned probe on voxel centres (pitch = h, dr = h): every sample
    hits a voxel centre, so the nearest index is known by hand and the
    trilinear HU reproduces the voxel value exactly."""
    rng = np.random.default_rng(3)
    shape = (30, 20, 16)
    lab = rng.integers(0, 5, shape).astype(np.uint8)
    hu = rng.integers(-1000, 2000, shape).astype(np.int16)
    probe = scene.linear_probe(8, 16, 16.0, 1.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (7.5, 9.0, 6.0))
    res = oracle.render_frame(lab, hu, 1.0, scene.tissue_table(), probe, scene.Options(), pose)
    for l in range(8):
        for s in range(16):
            i, j, k = 4 + l, 9, 6 + s      # x = l - 3.5 + 7.5
            assert res["nn_index"][l, s] == (k * 20 + j) * 16 + i
            assert res["label"][l, s] == lab[k, j, i]
            assert res["hu"][l, s] == hu[k, j, i]


def test_outside_volume_is_water():
    lab, hu = _homog((8, 8, 8), 3)
    probe = scene.linear_probe(4, 16, 16.0, 1.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (100.0, 100.0, 100.0))
    res = oracle.render_frame(lab, hu, 1.0, scene.tissue_table(), probe, scene.Options(), pose)
    assert np.all(res["nn_index"] == -1) and np.all(res["label"] == 0) and np.all(res["hu"] == 0)


def test_label_outside_table_is_an_error():
    lab, hu = _homog((8, 8, 8), 7)
    probe = scene.linear_probe(4, 16, 4.0, 1.0)
    pose = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (3.0, 3.0, 1.0))
    with pytest.raises(ValueError):
        oracle.render_frame(lab, hu, 1.0, scene.tissue_table(), probe, scene.Options(), pose)


def test_scan_conversion_inverts_the_fan():
    """Bilinear interpolation is exact on affine images, so ramps in the
    line and sample indices come back as the analytic fractional indices
    theta / dtheta + (NL-1)/2 and (rho - r0) / dr inside the fan; outside
    the fan the frame is 0."""
    probe = scene.curvilinear_probe(64, 128, 80.0, 60.0, 40.0, 65, 50)
    NL, NS = 64, 128
    dth = math.radians(60.0) / (NL - 1)
    dr = 80.0 / NS
    ramp_l = np.repeat(np.arange(NL, dtype=float)[:, None], NS, axis=1)
    ramp_s = np.repeat(np.arange(NS, dtype=float)[None, :], NL, axis=0)
    fl_img = oracle.scan_convert(probe, ramp_l)
    fs_img = oracle.scan_convert(probe, ramp_s + 1.0)
    half = math.radians(30.0)
    xmax = 120.0 * math.sin(half)
    zmin, zmax = 40.0 * math.cos(half), 120.0
    inside = 0
    for r in range(50):
        for c in range(65):
            x = -xmax + (c + 0.5) * 2 * xmax / 65
            z = zmin + (r + 0.5) * (zmax - zmin) / 50
            fl = math.atan2(x, z) / dth + (NL - 1) / 2
            fs = (math.hypot(x, z) - 40.0) / dr
            if 1e-9 < fl < NL - 1 - 1e-9 and 1e-9 < fs < NS - 1 - 1e-9:
                inside += 1
                assert abs(fl_img[r, c] - fl) < 1e-9
                assert abs(fs_img[r, c] - (fs + 1.0)) < 1e-9
            elif not (-1e-9 <= fl <= NL - 1 + 1e-9 and -1e-9 <= fs <= NS - 1 + 1e-9):
                assert fs_img[r, c] == 0.0
    assert inside > 500
    # the middle column (odd width) is the fan axis: theta = 0
    assert np.allclose(fl_img[fs_img[:, 32] > 0, 32], (NL - 1) / 2, atol=1e-12)


def _tiny_cases():
    rng = np.random.default_rng(21)
    shape = (12, 14, 16)
    lab = np.repeat(rng.integers(0, 5, (12, 14, 4)), 4, axis=2).astype(np.uint8)
    hu = rng.integers(-200, 800, shape).astype(np.int16)
    probes = [scene.linear_probe(6, 24, 12.0, 1.0, psf_sigma_ax_mm=0.6, psf_sigma_lat_mm=1.2),
              scene.curvilinear_probe(7, 20, 10.0, 40.0, 5.0, 9, 8, psf_sigma_ax_mm=0.5,
                                      psf_sigma_lat_mm=0.8)]
    poses = [np.array([[0.8, 0.6, 0, 7.3], [0, 0, -1, 12.1], [-0.6, 0.8, 0, 5.2]], np.float32),
             np.array([[0.36, 0.48, -0.8, 8.0], [0.8, -0.6, 0.0, 3.1], [-0.48, -0.64, -0.6, 10.7]],
                      np.float32)]
    for probe in probes:
        for pose in poses:
            for opt in (scene.Options(1, 1, 0, 1), scene.Options(2, 0, 1, 1), scene.Options(1, 1, 1, 0)):
                yield lab, hu, probe, pose, opt


def test_oracle_matches_brute_force():
    for lab, hu, probe, pose, opt in _tiny_cases():
        o = oracle.render_frame(lab, hu, 1.0, scene.tissue_table(), probe, opt, pose, env=3,
                                seed=0x1234567890, step=7)
        b = brute.render(lab, hu, 1.0, scene.tissue_table(), probe, opt, pose, env=3,
                         seed=0x1234567890, step=7)
        assert np.array_equal(o["nn_index"], b["nn_index"])
        assert np.array_equal(o["label"], b["label"])
        for k in ("hu", "E", "cos_theta", "S", "envelope", "logimg", "frame"):
            scale = max(np.abs(o[k]).max(), 1e-300)
            assert np.abs(o[k] - b[k]).max() <= 1e-12 * scale, k


def test_touched_voxels_small():
    lab, hu, probe, pose, _ = next(_tiny_cases())
    tot, per = oracle.touched_voxels([(lab, hu, 1.0)], [probe], np.zeros((1, 2), np.int32), pose[None])
    nz, ny, nx = lab.shape
    seen = set()
    for l in range(probe.n_lines):
        for s in range(probe.n_samples):
            u = oracle.sample_coords(probe, pose, 1.0, l, s)
            ni = [math.floor(float(np.float32(x + np.float32(0.5)))) for x in u]
            if 0 <= ni[0] < nx and 0 <= ni[1] < ny and 0 <= ni[2] < nz:
                seen.add((ni[0], ni[1], ni[2]))
            f = [math.floor(float(x)) for x in u]
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        q = (f[0] + dx, f[1] + dy, f[2] + dz)
                        if 0 <= q[0] < nx and 0 <= q[1] < ny and 0 <= q[2] < nz:
                            seen.add(q)
    assert tot == per[0] == len(seen)


def test_elevation_sweep_closed_forms():
    """The 3-D probe's elevation sweep (Sec. 4, Task 3; App. C: 5 planes
    10 mm apart): plane e of a pose is the pose moved by
    y_e = (e - (E - 1) / 2) * pitch along its own elevation axis (the
    rotation's y column), the rotation unchanged.  Checked on dyadic poses
    (exact in FP32) against hand-written translations."""
    ident = _axis_pose([(1, 0, 0), (0, 1, 0), (0, 0, 1)], (10.0, 20.0, 30.0))
    quarter = _axis_pose([(0, 1, 0), (0, 0, 1), (1, 0, 0)], (1.5, -2.25, 4.0))   # y axis along +z
    out = oracle.sweep_elevation(np.stack([ident, quarter]), 5, 10.0)
    assert out.shape == (10, 3, 4)
    for e in range(5):
        y = (e - 2) * 10.0
        np.testing.assert_array_equal(out[e, :, :3], ident[:, :3])
        np.testing.assert_array_equal(out[e, :, 3], [10.0, 20.0 + y, 30.0])
        np.testing.assert_array_equal(out[5 + e, :, :3], quarter[:, :3])
        np.testing.assert_array_equal(out[5 + e, :, 3], [1.5, -2.25, 4.0 + y])
    # an even count straddles the pose: offsets -1.5, -0.5, 0.5, 1.5 pitches
    out4 = oracle.sweep_elevation(ident[None], 4, 2.0)
    np.testing.assert_array_equal(out4[:, 1, 3], [17.0, 19.0, 21.0, 23.0])
    # one plane: the pose itself
    np.testing.assert_array_equal(oracle.sweep_elevation(quarter[None], 1, 7.0)[0], quarter)
