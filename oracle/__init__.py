"""CPU oracle for the model-based ultrasound render (SonoGym, App. B.2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, the smoke check and the
CPU-baseline leg of ``bench.py``; never by the product path.

* ``ussim_oracle.c`` (O1): FP64 C renderer, one frame at a time, OpenMP over
  frames for the CPU baseline.  Loaded here through ctypes; compiled on
  first use (or by ``build()``) with ``-ffp-contract=off``.
* ``brute.py`` (O2): pure-Python restatement on tiny inputs (direct sums,
  full 2-D PSF, its own Philox and Box-Muller).
* ``surrogate_ref.py`` (O3): PyTorch CPU float64 network / loss / optimiser
  reference of the learned surrogate.
* ``hist_match.py``: histogram matching of CT slices (the learned
  simulator's input), exact integer decisions.

Nothing here shares code with the CUDA path.  The synthetic inputs come
from ``paper_2507_01152_gb300.scene``, which holds none of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ussim_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libussim_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (FP32 index path must not be contracted)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class OrVolume(C.Structure):
    _fields_ = [("labels", C.c_void_p), ("hu", C.c_void_p), ("nx", C.c_int32),
                ("ny", C.c_int32), ("nz", C.c_int32), ("voxel_mm", C.c_float), ("id", C.c_int32)]


class OrTissue(C.Structure):
    _fields_ = [("alpha_db_cm_mhz", C.c_float), ("z_mrayl", C.c_float), ("mu0", C.c_float),
                ("sigma0", C.c_float), ("mu1", C.c_float)]


class OrProbe(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_lines", C.c_int32), ("n_samples", C.c_int32),
                ("depth_mm", C.c_float), ("pitch_mm", C.c_float), ("fan_deg", C.c_float),
                ("radius_mm", C.c_float), ("out_w", C.c_int32), ("out_h", C.c_int32),
                ("f_mhz", C.c_float), ("e0", C.c_float), ("psf_sigma_ax_mm", C.c_float),
                ("psf_sigma_lat_mm", C.c_float), ("dyn_range_db", C.c_float)]


class OrOptions(C.Structure):
    _fields_ = [("refl_power", C.c_int32), ("transmission", C.c_int32),
                ("z_mode", C.c_int32), ("speckle", C.c_int32), ("speckle_anchor", C.c_int32),
                ("speckle_levels", C.c_int32), ("speckle_cell_mm", C.c_float)]


class OrFrameOut(C.Structure):
    _fields_ = [("frame", C.c_void_p), ("envelope", C.c_void_p), ("logimg", C.c_void_p),
                ("S", C.c_void_p), ("T", C.c_void_p), ("E", C.c_void_p), ("cos_theta", C.c_void_p),
                ("hu", C.c_void_p), ("nn_index", C.c_void_p), ("label", C.c_void_p), ("n1", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.oracle_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.oracle_speckle_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                               C.c_uint32, C.c_void_p]
            L.oracle_n0.argtypes = [C.c_void_p, C.c_uint32]
            L.oracle_n0.restype = C.c_double
            L.oracle_n1_threshold.argtypes = [C.c_double]
            L.oracle_n1_threshold.restype = C.c_uint64
            L.oracle_psf_taps.argtypes = [C.c_double, C.c_double, C.c_void_p, C.c_int]
            L.oracle_psf_taps.restype = C.c_int
            L.oracle_scan_convert.argtypes = [C.POINTER(OrProbe), C.c_void_p, C.c_void_p]
            L.oracle_render_frame.argtypes = [C.POINTER(OrVolume), C.POINTER(OrTissue), C.c_int,
                                              C.POINTER(OrProbe), C.POINTER(OrOptions), C.c_void_p,
                                              C.c_uint32, C.c_uint64, C.c_uint64,
                                              C.POINTER(OrFrameOut)]
            L.oracle_render_frame.restype = C.c_int
            L.oracle_render_batch.argtypes = [C.POINTER(OrVolume), C.c_int, C.POINTER(OrTissue),
                                              C.c_int, C.POINTER(OrProbe), C.c_int,
                                              C.POINTER(OrOptions), C.c_void_p, C.c_int, C.c_void_p,
                                              C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p,
                                              C.c_int]
            L.oracle_render_batch.restype = C.c_int
            L.oracle_touched_voxels.argtypes = [C.POINTER(OrVolume), C.c_int, C.POINTER(OrProbe),
                                                C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            L.oracle_touched_voxels.restype = C.c_int64
            L.oracle_sample_coords.argtypes = [C.POINTER(OrProbe), C.c_void_p, C.c_float, C.c_int,
                                               C.c_int, C.c_void_p]
            L.oracle_sample_slice.argtypes = [C.POINTER(OrVolume), C.POINTER(OrProbe), C.c_void_p, C.c_void_p]
            L.oracle_sample_slice.restype = C.c_int
            L.oracle_sample_slice_raw.argtypes = [C.POINTER(OrVolume), C.POINTER(OrProbe), C.c_void_p, C.c_void_p]
            L.oracle_sample_slice_raw.restype = C.c_int
            L.oracle_sample_slice_grid.argtypes = [C.POINTER(OrVolume), C.POINTER(OrProbe), C.c_void_p, C.c_int,
                                                   C.c_int, C.c_void_p]
            L.oracle_sample_slice_grid.restype = C.c_int
            L.oracle_anchored_noise.argtypes = [C.c_void_p, C.c_int32, C.c_float, C.c_uint32, C.c_uint64,
                                                C.c_void_p]
            L.oracle_recon_keep_threshold.argtypes = [C.c_double]
            L.oracle_recon_keep_threshold.restype = C.c_uint32
            L.oracle_recon_update.argtypes = [C.POINTER(OrVolume), C.POINTER(OrProbe), C.c_void_p, C.c_uint32,
                                              C.c_uint64, C.c_uint64, C.c_int32, C.c_double, C.c_void_p,
                                              C.c_void_p]
            L.oracle_recon_update.restype = C.c_int64
            L.oracle_recon_observe.argtypes = [C.POINTER(OrVolume), C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- marshalling

def or_probe(p) -> OrProbe:
    return OrProbe(p.kind, p.n_lines, p.n_samples, p.depth_mm, p.pitch_mm, p.fan_deg,
                   p.radius_mm, p.out_w, p.out_h, p.f_mhz, p.e0, p.psf_sigma_ax_mm,
                   p.psf_sigma_lat_mm, p.dyn_range_db)


def or_table(table):
    arr = (OrTissue * len(table))()
    for i, t in enumerate(table):
        arr[i] = OrTissue(t.alpha_db_cm_mhz, t.z_mrayl, t.mu0, t.sigma0, t.mu1)
    return arr


def or_options(o) -> OrOptions:
    return OrOptions(o.refl_power, o.transmission, o.z_mode, o.speckle, getattr(o, "speckle_anchor", 0),
                     getattr(o, "speckle_levels", 1), getattr(o, "speckle_cell_mm", 0.25))


class _Vol:
    """Keeps the numpy arrays alive next to the ctypes descriptor."""

    def __init__(self, labels, hu, voxel_mm, vol_id=0):
        self.labels = np.ascontiguousarray(labels, np.uint8)
        self.hu = np.ascontiguousarray(hu, np.int16)
        nz, ny, nx = self.labels.shape
        self.desc = OrVolume(self.labels.ctypes.data, self.hu.ctypes.data, nx, ny, nz, voxel_mm, vol_id)


# --------------------------------------------------------------------- API

def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def speckle_words(seed, step, env, line, sample):
    out = np.zeros(4, np.uint32)
    lib().oracle_speckle_words(seed, step, env, line, sample, _ptr(out))
    return out


def n0(words, sample):
    w = np.asarray(words, np.uint32)
    return lib().oracle_n0(_ptr(w), sample)


def n1_threshold(mu1):
    return int(lib().oracle_n1_threshold(float(mu1)))


def psf_taps(sigma_mm, spacing_mm, max_taps=4096):
    t = np.zeros(max_taps)
    K = lib().oracle_psf_taps(sigma_mm, spacing_mm, _ptr(t), max_taps)
    if K < 0:
        raise ValueError("too many taps")
    return t[:2 * K + 1].copy()


def sample_coords(probe, pose, voxel_mm, line, sample):
    u = np.zeros(3, np.float32)
    pr = or_probe(probe)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    lib().oracle_sample_coords(C.byref(pr), _ptr(M), voxel_mm, line, sample, _ptr(u))
    return u


def scan_convert(probe, logimg):
    pr = or_probe(probe)
    y = np.ascontiguousarray(logimg, np.float64)
    out = np.zeros((probe.out_h, probe.out_w), np.float64)
    lib().oracle_scan_convert(C.byref(pr), _ptr(y), _ptr(out))
    return out


def render_frame(labels, hu, voxel_mm, table, probe, options, pose, env=0, seed=0, step=0, vol_id=0):
    """Render one frame; returns a dict of every export (numpy arrays;
    "envelope" is I = P (x) R_imp + E (P (x) T) before the log, "S" the image
    under an identity PSF (R_imp + E T), "T" the scatter pattern, "E" the
    energy; "n1" holds the anchored scatter map N1 per sample, NaN in the
    beam-keyed mode)."""
    vol = _Vol(labels, hu, voxel_mm, vol_id)
    NL, NS = probe.n_lines, probe.n_samples
    res = {
        "frame": np.zeros((probe.out_h, probe.out_w)),
        "envelope": np.zeros((NL, NS)), "logimg": np.zeros((NL, NS)), "S": np.zeros((NL, NS)),
        "T": np.zeros((NL, NS)),
        "E": np.zeros((NL, NS)), "cos_theta": np.zeros((NL, NS)), "hu": np.zeros((NL, NS)),
        "nn_index": np.zeros((NL, NS), np.int32), "label": np.zeros((NL, NS), np.uint8),
        "n1": np.full((NL, NS), np.nan),
    }
    o = OrFrameOut(*[res[k].ctypes.data for k in
                     ("frame", "envelope", "logimg", "S", "T", "E", "cos_theta", "hu", "nn_index", "label",
                      "n1")])
    tab = or_table(table)
    pr = or_probe(probe)
    op = or_options(options)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    rc = lib().oracle_render_frame(C.byref(vol.desc), tab, len(table), C.byref(pr), C.byref(op),
                                   _ptr(M), env, seed, step, C.byref(o))
    if rc != 0:
        raise ValueError(f"oracle_render_frame failed: {rc}")
    return res


def render_batch(volumes, table, probes, options, envs, poses, seed, step, n_threads=1):
    """Render a batch.  volumes: list of (labels, hu, voxel_mm); envs int32
    [B][2]; poses float32 [B][3][4].  Returns (frames float64 flat, offsets)."""
    vols = [_Vol(l, h, v, i) for i, (l, h, v) in enumerate(volumes)]
    vd = (OrVolume * len(vols))(*[v.desc for v in vols])
    pd = (OrProbe * len(probes))(*[or_probe(p) for p in probes])
    envs = np.ascontiguousarray(envs, np.int32)
    B = envs.shape[0]
    sizes = np.array([probes[e[1]].out_h * probes[e[1]].out_w for e in envs], np.int64)
    offsets = np.zeros(B + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    frames = np.zeros(int(offsets[-1]), np.float64)
    P = np.ascontiguousarray(poses, np.float32).reshape(B, 12)
    op = or_options(options)
    rc = lib().oracle_render_batch(vd, len(vols), or_table(table), len(table), pd, len(probes),
                                   C.byref(op), _ptr(envs), B, _ptr(P), seed, step,
                                   _ptr(frames), _ptr(offsets), n_threads)
    if rc != 0:
        raise ValueError(f"oracle_render_batch failed: {rc}")
    return frames, offsets


def touched_voxels(volumes, probes, envs, poses):
    """(union count over the batch, per-frame counts) of voxels read."""
    vols = [_Vol(l, h, v) for (l, h, v) in volumes]
    vd = (OrVolume * len(vols))(*[v.desc for v in vols])
    pd = (OrProbe * len(probes))(*[or_probe(p) for p in probes])
    envs = np.ascontiguousarray(envs, np.int32)
    B = envs.shape[0]
    per = np.zeros(B, np.int64)
    P = np.ascontiguousarray(poses, np.float32).reshape(B, 12)
    tot = lib().oracle_touched_voxels(vd, len(vols), pd, _ptr(envs), B, _ptr(P), _ptr(per))
    return int(tot), per


def anchored_noise(pos, levels, cell_mm, vol_id, seed):
    """(N0, N1) of the volume-anchored multi-scale scatter maps at a
    volume-frame position (mm, float32)"""
    p = np.ascontiguousarray(pos, np.float32)
    out = np.zeros(2)
    lib().oracle_anchored_noise(_ptr(p), levels, cell_mm, vol_id, seed, _ptr(out))
    return float(out[0]), float(out[1])


def recon_update(labels, hu, voxel_mm, probe, pose, env, seed, step, bone_label, p_miss, recon):
    """add one frame's kept bone-surface points to `recon` (uint8 volume,
    updated in place); returns (ground-truth points, kept points)"""
    vol = _Vol(labels, hu, voxel_mm)
    pr = or_probe(probe)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    assert recon.dtype == np.uint8 and recon.flags.c_contiguous and recon.shape == vol.labels.shape
    kept = C.c_int64(0)
    n = lib().oracle_recon_update(C.byref(vol.desc), C.byref(pr), _ptr(M), env, seed, step, bone_label,
                                  float(p_miss), _ptr(recon), C.byref(kept))
    return int(n), int(kept.value)


def recon_observe(recon, voxel_mm, pose):
    """the reconstruction voxelized in the probe frame: uint8 [40][40][40] (h, w, e)"""
    nz, ny, nx = recon.shape
    desc = OrVolume(None, None, nx, ny, nz, voxel_mm, 0)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    obs = np.zeros((40, 40, 40), np.uint8)
    lib().oracle_recon_observe(C.byref(desc), _ptr(np.ascontiguousarray(recon, np.uint8)), _ptr(M), _ptr(obs))
    return obs


def recon_keep_threshold(p_miss):
    return int(lib().oracle_recon_keep_threshold(float(p_miss)))


def sample_slice(labels, hu, voxel_mm, probe, pose):
    """surrogate input of one env: [out_h][out_w][3] = (label / 4,
    clamp(HU / 1000, -1, 3), inside-fan flag)"""
    vol = _Vol(labels, hu, voxel_mm)
    out = np.zeros((probe.out_h, probe.out_w, 3))
    pr = or_probe(probe)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    lib().oracle_sample_slice(C.byref(vol.desc), C.byref(pr), _ptr(M), _ptr(out))
    return out


def sample_slice_raw(labels, hu, voxel_mm, probe, pose):
    """[out_h][out_w][3] = (label, trilinear HU (unscaled, FP64), inside-fan
    flag) on one env's output pixel grid"""
    vol = _Vol(labels, hu, voxel_mm)
    out = np.zeros((probe.out_h, probe.out_w, 3))
    pr = or_probe(probe)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    lib().oracle_sample_slice_raw(C.byref(vol.desc), C.byref(pr), _ptr(M), _ptr(out))
    return out


def sweep_elevation(poses, n_elev, pitch_mm):
    """Elevation sweep of the 3-D probe (Sec. 4, Task 3: volumetric images
    H x W x E; App. C: E = 5 planes 10 mm apart).  Plane e of pose b is the
    pose moved along its own elevation axis (the rotation's y column) by
    y_e = (e - (E - 1) / 2) * pitch: t' = t + R[:, 1] * y_e.  FP32 with one
    rounding per product and per sum, pose by pose and plane by plane;
    entry b * E + e of the result."""
    P = np.asarray(poses, np.float32).reshape(-1, 3, 4)
    out = np.zeros((len(P) * n_elev, 3, 4), np.float32)
    for b in range(len(P)):
        for e in range(n_elev):
            y = np.float32(np.float32(e - 0.5 * (n_elev - 1)) * np.float32(pitch_mm))
            M = P[b].copy()
            for r in range(3):
                M[r, 3] = np.float32(P[b, r, 3] + np.float32(P[b, r, 1] * y))
            out[b * n_elev + e] = M
    return out


def sample_slice_grid(labels, hu, voxel_mm, probe, pose, H, W):
    """surrogate input of one env on an H x W grid over its output field:
    [H][W][3] = (label / 4, clamp(HU / 1000, -1, 3), inside-field flag)"""
    vol = _Vol(labels, hu, voxel_mm)
    out = np.zeros((H, W, 3))
    pr = or_probe(probe)
    M = np.ascontiguousarray(pose, np.float32).reshape(12)
    lib().oracle_sample_slice_grid(C.byref(vol.desc), C.byref(pr), _ptr(M), H, W, _ptr(out))
    return out


def fan_mask(probe):
    """[out_h][out_w] 1 where an output pixel centre lies inside the fan (the
    scan conversion's test, FP64); all ones for a linear probe"""
    H, W = probe.out_h, probe.out_w
    if probe.kind == 0:
        return np.ones((H, W), bool)
    NL, NS = probe.n_lines, probe.n_samples
    f32 = lambda v: float(np.float32(v))
    r0, D = f32(probe.radius_mm), f32(probe.depth_mm)
    half = 0.5 * f32(probe.fan_deg) * np.pi / 180.0
    dth = f32(probe.fan_deg) * np.pi / 180.0 / (NL - 1)
    dr = D / NS
    xmax = (r0 + D) * np.sin(half)
    zmin, zmax = r0 * np.cos(half), r0 + D
    m = np.zeros((H, W), bool)
    for r in range(H):
        z = zmin + (r + 0.5) * (zmax - zmin) / H
        for c in range(W):
            x = -xmax + (c + 0.5) * 2 * xmax / W
            fl = np.arctan2(x, z) / dth + 0.5 * (NL - 1)
            fs = (np.hypot(x, z) - r0) / dr
            m[r, c] = 0 <= fl <= NL - 1 and 0 <= fs <= NS - 1
    return m


def resize_frame(src, probe, mask=None):
    """An H x W frame over a probe's output field onto the probe's own
    out_h x out_w grid: output pixel (r, c) reads src at
    fy = (r + 1/2) H / out_h - 1/2, fx = (c + 1/2) W / out_w - 1/2 (pixel
    centres of the same field), clamped to the source, bilinearly; 0 outside
    a curvilinear fan (mask = fan_mask(probe), computed if not given)."""
    src = np.asarray(src, np.float64)
    H, W = src.shape
    OH, OW = probe.out_h, probe.out_w
    if mask is None:
        mask = fan_mask(probe)
    out = np.zeros((OH, OW))
    for r in range(OH):
        fy = min(max((r + 0.5) * H / OH - 0.5, 0.0), H - 1.0)
        y0 = min(int(np.floor(fy)), H - 2)
        a = fy - y0
        for c in range(OW):
            if not mask[r, c]:
                continue
            fx = min(max((c + 0.5) * W / OW - 0.5, 0.0), W - 1.0)
            x0 = min(int(np.floor(fx)), W - 2)
            b = fx - x0
            top = src[y0, x0] + b * (src[y0, x0 + 1] - src[y0, x0])
            bot = src[y0 + 1, x0] + b * (src[y0 + 1, x0 + 1] - src[y0 + 1, x0])
            out[r, c] = top + a * (bot - top)
    return out


def audit_selected(B, seed, step, fraction, score, threshold):
    """The gate's physics audit: env b is audited when the gate keeps it
    (not score[b] > threshold) and word 0 of Philox-4x32-10 on counter
    (0, 0, b, 2), key (seed_lo ^ (uint32)(step * 0x9E3779B9), seed_hi), is
    below floor(fraction 2^32).  Returns a bool array [B]."""
    t = int(np.floor(fraction * 4294967296.0))
    key = [(seed & 0xFFFFFFFF) ^ ((step * 0x9E3779B9) & 0xFFFFFFFF), (seed >> 32) & 0xFFFFFFFF]
    out = np.zeros(B, bool)
    for b in range(B):
        if score[b] > threshold:
            continue
        out[b] = int(philox4x32_10([0, 0, b, 2], key)[0]) < t
    return out
