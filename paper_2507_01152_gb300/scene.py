"""Seeded synthetic inputs for the ultrasound render path.

This module holds no step of the simulation method: it only draws the
inputs that both the CUDA path and the CPU oracle consume.

* spine-like label + HU volumes (stand-ins for the CT label maps and CT
  volumes of the paper's patient models, Sec. 4 "Assets");
* the synthetic tissue table (the paper takes its per-tissue constants from a
  commercial simulator and does not print them, App. B.2);
* probe descriptors (linear 200x150 at 0.5 mm as in App. C.1, and the
  curvilinear probes of the batched workloads);
* probe poses on the dorsal skin, and seeded random walks of them.

Volumes are numpy arrays indexed ``[k][j][i]`` (x = i fastest), voxel
``(i, j, k)`` centred at ``(i, j, k) * h`` mm.  Axes: i left-right,
j anterior -> posterior (dorsal skin at high j), k cranio-caudal.
Poses are float32 ``[3][4]`` matrices ``[R | t]`` mapping probe-frame mm
(x lateral, y elevation, z depth along the beam) to volume-frame mm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# label ids of the synthetic tissue classes
WATER, SKIN, FAT, MUSCLE, BONE = 0, 1, 2, 3, 4

# class-mean HU (water, skin, fat, muscle, bone)
HU_MEAN = np.array([0.0, 30.0, -100.0, 50.0, 700.0])


@dataclass(frozen=True)
class Tissue:
    """Raw per-tissue settings, in the units they are usually quoted in."""
    alpha_db_cm_mhz: float   # attenuation, dB / (cm MHz)
    z_mrayl: float           # acoustic impedance, MRayl
    mu0: float               # scatter mean
    sigma0: float            # scatter std
    mu1: float               # scatter density threshold on N1 (N1 <= mu1)


def tissue_table() -> list[Tissue]:
    """Synthetic tissue table, index = label.

    Our own plausible values, not the paper's (which are not printed).
    Water never scatters: mu1 = -inf makes the density test always fail.
    """
    return [
        Tissue(0.002, 1.48, 0.0, 0.0, -math.inf),  # water / background / gel
        Tissue(0.6, 1.60, 0.5, 0.2, 0.5),          # skin shell
        Tissue(0.5, 1.38, 0.3, 0.15, 0.3),         # fat
        Tissue(1.1, 1.70, 0.5, 0.2, 0.6),          # muscle
        Tissue(20.0, 7.80, 0.8, 0.3, 0.8),         # bone
    ]


@dataclass(frozen=True)
class Probe:
    """Probe descriptor.  kind 0 = linear, 1 = curvilinear.

    Linear: lines at lateral offsets (l - (NL-1)/2) * pitch, samples at
    depth s * depth/NS, output image NS rows x NL columns.
    Curvilinear: apex r0 behind the face, fan angle ``fan_deg`` over NL
    lines, samples at radius r0 + s * depth/NS, scan-converted to
    out_h x out_w.
    """
    kind: int
    n_lines: int
    n_samples: int
    depth_mm: float
    pitch_mm: float = 0.0
    fan_deg: float = 0.0
    radius_mm: float = 0.0
    out_w: int = 0
    out_h: int = 0
    f_mhz: float = 5.0
    e0: float = 1.0
    psf_sigma_ax_mm: float = 0.3
    psf_sigma_lat_mm: float = 1.0
    dyn_range_db: float = 60.0

    def as_dict(self):
        return asdict(self)


def linear_probe(n_lines=128, n_samples=256, depth_mm=80.0, pitch_mm=0.5, **kw) -> Probe:
    return Probe(kind=0, n_lines=n_lines, n_samples=n_samples, depth_mm=depth_mm,
                 pitch_mm=pitch_mm, out_w=n_lines, out_h=n_samples, **kw)


def curvilinear_probe(n_lines=256, n_samples=512, depth_mm=80.0, fan_deg=60.0,
                      radius_mm=40.0, out_w=256, out_h=256, **kw) -> Probe:
    return Probe(kind=1, n_lines=n_lines, n_samples=n_samples, depth_mm=depth_mm,
                 fan_deg=fan_deg, radius_mm=radius_mm, out_w=out_w, out_h=out_h, **kw)


@dataclass(frozen=True)
class Options:
    """Model switches.

    refl_power: exponent p of the reflection term (1 = paper, 2 = squared
    reflection coefficient).  transmission: 1 adds the interface
    transmission loss ln(1 - r^2) to the energy, 0 is attenuation only
    (paper).  z_mode: 0 = impedance from HU, 1 = impedance from the tissue
    table.  speckle: 1 = random scatter pattern, 0 = scatter fixed at mu0.
    speckle_anchor: 0 = scatter maps keyed by (env, line, sample, step);
    1 = fixed maps over the volume (they move with the tissue), with
    speckle_levels scales (1-3) of cells of edge speckle_cell_mm * 2^k.
    volume_layout: memory layout of the HU grid on the GPU (0 = corner
    records, 1 = the grid as given); it does not change the images.
    """
    refl_power: int = 1
    transmission: int = 1
    z_mode: int = 0
    speckle: int = 1
    speckle_anchor: int = 0
    speckle_levels: int = 1
    speckle_cell_mm: float = 0.25
    volume_layout: int = 0


# --------------------------------------------------------------------------
# volumes
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class VolumeSpec:
    nx: int
    ny: int
    nz: int
    voxel_mm: float
    n_vertebrae: int
    seed: int
    hu_noise: float = 20.0


def _smooth_noise_2d(rng, n_a, n_b, out_a, out_b):
    """Low-frequency field on an (out_a, out_b) grid, values in [0, 1]."""
    coarse = rng.random((n_a + 1, n_b + 1))
    ia = np.linspace(0, n_a, out_a)
    ib = np.linspace(0, n_b, out_b)
    a0 = np.minimum(ia.astype(int), n_a - 1)
    b0 = np.minimum(ib.astype(int), n_b - 1)
    fa = (ia - a0)[:, None]
    fb = (ib - b0)[None, :]
    c00 = coarse[a0][:, b0]
    c10 = coarse[a0 + 1][:, b0]
    c01 = coarse[a0][:, b0 + 1]
    c11 = coarse[a0 + 1][:, b0 + 1]
    # smoothstep blend
    fa = fa * fa * (3 - 2 * fa)
    fb = fb * fb * (3 - 2 * fb)
    return (c00 * (1 - fa) * (1 - fb) + c10 * fa * (1 - fb)
            + c01 * (1 - fa) * fb + c11 * fa * fb)


def body_geometry(spec: VolumeSpec):
    """Centre and semi-axes (mm) of the elliptic body cross-section."""
    X, Y = spec.nx * spec.voxel_mm, spec.ny * spec.voxel_mm
    h = spec.voxel_mm
    cx, cy = 0.5 * (spec.nx - 1) * h, 0.5 * (spec.ny - 1) * h
    return cx, cy, 0.42 * X, 0.38 * Y


def make_volume(spec: VolumeSpec):
    """Spine-like label + HU volume.

    Elliptic body along k with a 2 mm skin shell, a fat layer 8-15 mm thick
    (seeded smooth thickness), muscle inside, and a chain of vertebrae
    (unions of ellipsoids: body, arch, spinous process, two transverse
    processes) whose spinous tips sit 25-40 mm under the dorsal skin.
    Returns (labels uint8 [nz][ny][nx], hu int16 [nz][ny][nx]).
    """
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    nx, ny, nz, h = spec.nx, spec.ny, spec.nz, spec.voxel_mm
    X, Y, Z = nx * h, ny * h, nz * h
    cx, cy, ax, ay = body_geometry(spec)
    sc = min(1.0, min(X, Y) / 200.0)          # vertebra size scale

    # fat thickness over (angle, k): 8..15 mm
    n_ang = 256
    fat_field = 8.0 + 7.0 * _smooth_noise_2d(rng, 6, 4, n_ang, nz)

    # vertebra centres along k
    n = spec.n_vertebrae
    spacing = Z / (n + 0.5)
    zc = (np.arange(n) + 0.75) * spacing + rng.uniform(-2.0, 2.0, n)
    tip_depth = rng.uniform(25.0, 40.0, n) * max(sc, 0.75)
    parts = []   # (centre xyz, semi-axes xyz)
    for v in range(n):
        y_tip = cy + ay - tip_depth[v]
        z0 = zc[v]
        s = sc
        parts += [
            ((cx, y_tip - 12 * s, z0), (3.0 * s, 12.0 * s, 5.0 * s)),      # spinous process
            ((cx, y_tip - 27 * s, z0), (14.0 * s, 5.0 * s, 6.0 * s)),      # arch / lamina
            ((cx - 20 * s, y_tip - 29 * s, z0), (11.0 * s, 4.0 * s, 4.0 * s)),  # transverse L
            ((cx + 20 * s, y_tip - 29 * s, z0), (11.0 * s, 4.0 * s, 4.0 * s)),  # transverse R
            ((cx, y_tip - 52 * s, z0), (18.0 * s, 13.0 * s, 10.0 * s)),    # vertebral body
        ]

    x = (np.arange(nx) * h).astype(np.float32)
    y = (np.arange(ny) * h).astype(np.float32)
    dx = (x - cx)[None, :]
    dy = (y - cy)[:, None]
    rho_n = np.sqrt((dx / ax) ** 2 + (dy / ay) ** 2)                 # [ny][nx]
    ang = np.arctan2(dy / ay, dx / ax)
    # radius of the ellipse along this direction, and inward depth
    r_loc = 1.0 / np.sqrt((np.cos(ang) / ax) ** 2 + (np.sin(ang) / ay) ** 2)
    depth_in = (1.0 - rho_n) * r_loc                                  # mm under the skin
    ang_idx = ((ang + np.pi) / (2 * np.pi) * (n_ang - 1)).round().astype(int)

    labels = np.zeros((nz, ny, nx), np.uint8)
    inside = rho_n <= 1.0
    skin = inside & (depth_in < 2.0)
    for k in range(nz):
        fat_t = fat_field[ang_idx, k]
        sl = np.full((ny, nx), WATER, np.uint8)
        sl[inside] = MUSCLE
        sl[inside & (depth_in < 2.0 + fat_t)] = FAT
        sl[skin] = SKIN
        labels[k] = sl

    zz = (np.arange(nz) * h)
    for (pc, pa) in parts:
        lo = [max(0, int(math.floor((pc[d] - pa[d]) / h))) for d in range(3)]
        hi = [min(m, int(math.ceil((pc[d] + pa[d]) / h)) + 1) for d, m in enumerate((nx, ny, nz))]
        if any(l >= u for l, u in zip(lo, hi)):
            continue
        ex = ((x[lo[0]:hi[0]] - pc[0]) / pa[0]) ** 2
        ey = ((y[lo[1]:hi[1]] - pc[1]) / pa[1]) ** 2
        ez = ((zz[lo[2]:hi[2]] - pc[2]) / pa[2]) ** 2
        m = (ez[:, None, None] + ey[None, :, None] + ex[None, None, :]) <= 1.0
        m &= inside[None, lo[1]:hi[1], lo[0]:hi[0]]
        sub = labels[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[m] = BONE

    hu = np.empty((nz, ny, nx), np.int16)
    for k0 in range(0, nz, 16):
        k1 = min(nz, k0 + 16)
        lab = labels[k0:k1]
        v = HU_MEAN[lab] + rng.normal(0.0, spec.hu_noise, lab.shape)
        hu[k0:k1] = np.clip(np.rint(v), -1024, 3071).astype(np.int16)
    return labels, hu


# --------------------------------------------------------------------------
# poses
# --------------------------------------------------------------------------

def _rot(axis, ang):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def _frame_at(spec: VolumeSpec, dx_mm, k_mm, tilt_a, tilt_b, spin):
    """Probe pose on the dorsal skin: position, beam tilted about both
    tangents, rotated in-plane by ``spin`` about the beam."""
    cx, cy, ax, ay = body_geometry(spec)
    dx = float(np.clip(dx_mm, -0.95 * ax, 0.95 * ax))
    y = cy + ay * math.sqrt(max(0.0, 1.0 - (dx / ax) ** 2))
    p = np.array([cx + dx, y, k_mm])
    n = -np.array([dx / ax ** 2, (y - cy) / ay ** 2, 0.0])
    n /= np.linalg.norm(n)                        # inward normal (beam)
    t1 = np.array([0.0, 0.0, 1.0])                # cranio-caudal tangent
    t2 = np.cross(n, t1)
    t2 /= np.linalg.norm(t2)
    beam = _rot(t1, tilt_a) @ (_rot(t2, tilt_b) @ n)
    lat0 = np.cross(t1, beam)
    lat0 /= np.linalg.norm(lat0)
    lat = _rot(beam, spin) @ lat0
    elev = np.cross(beam, lat)
    R = np.stack([lat, elev, beam], axis=1)       # columns: probe x, y, z
    M = np.concatenate([R, p[:, None]], axis=1)
    return M


def dorsal_poses(spec: VolumeSpec, B: int, seed: int, tilt_deg=15.0,
                 half_width_mm=40.0, k_margin_mm=20.0) -> np.ndarray:
    """B poses uniform over the dorsal skin patch: |lateral offset| <=
    half_width_mm, k inside a margin, beam = inward normal tilted U(+-tilt)
    about both tangents, in-plane rotation U[0, pi).  float32 [B][3][4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = spec.nz * spec.voxel_mm
    out = np.empty((B, 3, 4), np.float32)
    t = math.radians(tilt_deg)
    for b in range(B):
        out[b] = _frame_at(spec, rng.uniform(-half_width_mm, half_width_mm),
                           rng.uniform(k_margin_mm, Z - k_margin_mm),
                           rng.uniform(-t, t), rng.uniform(-t, t),
                           rng.uniform(0.0, math.pi))
    return out


def midline_pose(spec: VolumeSpec) -> np.ndarray:
    """Probe centred on the dorsal midline, beam along -j, lines along i."""
    cx, cy, ax, ay = body_geometry(spec)
    h = spec.voxel_mm
    kc = 0.5 * (spec.nz - 1) * h
    # columns: lateral = +i, elevation = +k, beam = -j
    R = np.stack([np.array([1.0, 0, 0]), np.array([0, 0, 1.0]), np.array([0, -1.0, 0])], axis=1)
    t = np.array([cx, cy + ay, kc])
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


def random_walk_poses(spec: VolumeSpec, B: int, steps: int, seed: int,
                      step_mm=2.0, step_deg=2.0, tilt_deg=15.0,
                      half_width_mm=40.0, k_margin_mm=20.0) -> np.ndarray:
    """Per-env random walks over the dorsal skin: each step moves 2 mm
    along the skin and turns the probe by 2 degrees, re-projected onto the
    skin.  float32 [steps][B][3][4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = spec.nz * spec.voxel_mm
    t = math.radians(tilt_deg)
    st = np.empty((B, 5))
    st[:, 0] = rng.uniform(-half_width_mm, half_width_mm, B)
    st[:, 1] = rng.uniform(k_margin_mm, Z - k_margin_mm, B)
    st[:, 2] = rng.uniform(-t, t, B)
    st[:, 3] = rng.uniform(-t, t, B)
    st[:, 4] = rng.uniform(0.0, math.pi, B)
    out = np.empty((steps, B, 3, 4), np.float32)
    d = math.radians(step_deg)
    for s in range(steps):
        for b in range(B):
            out[s, b] = _frame_at(spec, *st[b])
        heading = rng.uniform(0, 2 * math.pi, B)
        st[:, 0] = np.clip(st[:, 0] + step_mm * np.cos(heading), -half_width_mm, half_width_mm)
        st[:, 1] = np.clip(st[:, 1] + step_mm * np.sin(heading), k_margin_mm, Z - k_margin_mm)
        which = rng.integers(0, 3, B)
        sign = rng.choice([-1.0, 1.0], B)
        for b in range(B):
            j = 2 + which[b]
            st[b, j] += sign[b] * d
        st[:, 2] = np.clip(st[:, 2], -t, t)
        st[:, 3] = np.clip(st[:, 3], -t, t)
    return out


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    """A set of volumes, probes, envs (volume_id, probe_id) and poses."""
    name: str
    volumes: list              # list of (VolumeSpec, labels, hu)
    probes: list               # list of Probe
    envs: np.ndarray           # int32 [B][2] (volume_id, probe_id)
    poses: np.ndarray          # float32 [B][3][4] or [steps][B][3][4]
    options: Options = field(default_factory=Options)
    seed: int = 0


def c1_spec():
    return VolumeSpec(128, 128, 128, 1.0, 2, 1000)


def c2_spec():
    return VolumeSpec(256, 256, 256, 0.5, 5, 1000)


def c3_specs():
    return [VolumeSpec(512, 512, 256, 0.5, 5, 1000 + v) for v in range(4)]


def c3_probes():
    return [linear_probe(128, 256, 80.0, 0.5),
            curvilinear_probe(192, 384, 80.0, 60.0, 40.0, 192, 192),
            curvilinear_probe(256, 512, 80.0, 60.0, 40.0, 256, 256)]


def workload_c1():
    """1 env, 128^3 at 1 mm, 2 vertebrae, linear 128 x 256 to 80 mm."""
    spec = c1_spec()
    lab, hu = make_volume(spec)
    return Workload("c1_single_linear_128x256", [(spec, lab, hu)], [linear_probe()],
                    np.zeros((1, 2), np.int32), midline_pose(spec)[None], seed=0x5EED0001)


def workload_c2(B=64, steps=None):
    """B envs on one 256^3 volume at 0.5 mm, curvilinear 256 x 512 -> 256 x 256."""
    spec = c2_spec()
    lab, hu = make_volume(spec)
    if steps is None:
        poses = dorsal_poses(spec, B, 2000)
    else:
        poses = random_walk_poses(spec, B, steps, 2000)
    return Workload(f"c2_batched_curvilinear_{B}env", [(spec, lab, hu)], [curvilinear_probe()],
                    np.zeros((B, 2), np.int32), poses, seed=0x5EED0002)


def workload_c3(B=512, steps=100, volumes=None):
    """B envs over 4 volumes of 512 x 512 x 256; env b uses volume b % 4 and
    probe b % 3 (linear 128 x 256, curvilinear 192 x 384, curvilinear
    256 x 512); seeded random-walk poses over ``steps`` steps."""
    specs = c3_specs()
    if volumes is None:
        volumes = [(s, *make_volume(s)) for s in specs]
    envs = np.stack([np.arange(B) % 4, np.arange(B) % 3], axis=1).astype(np.int32)
    poses = np.empty((steps, B, 3, 4), np.float32)
    for v in range(4):
        idx = np.nonzero(envs[:, 0] == v)[0]
        pw = random_walk_poses(specs[v], len(idx), steps, 3000 + v)
        poses[:, idx] = pw
    return Workload(f"c3_uneven_{B}env", volumes, c3_probes(), envs, poses, seed=0x5EED0003)


def workload_c5(B=1024, steps=3, volumes=None):
    """B envs over the four 512 x 512 x 256 volumes and three probes of C3,
    grouped by probe (the first third linear 128 x 256, the next
    curvilinear 192 x 384, the last curvilinear 256 x 512, so that the frames
    of one probe type are contiguous in the frame layout); env b uses volume
    b % 4; seeded random-walk poses over ``steps`` steps."""
    specs = c3_specs()
    if volumes is None:
        volumes = [(s, *make_volume(s)) for s in specs]
    probe_of = np.minimum(np.arange(B) * 3 // B, 2)
    envs = np.stack([np.arange(B) % 4, probe_of], axis=1).astype(np.int32)
    poses = np.empty((steps, B, 3, 4), np.float32)
    for v in range(4):
        idx = np.nonzero(envs[:, 0] == v)[0]
        poses[:, idx] = random_walk_poses(specs[v], len(idx), steps, 3100 + v)
    return Workload(f"c5_mixed_{B}env", volumes, c3_probes(), envs, poses, seed=0x5EED0005)


def workload_paper_replica(B=100):
    """100 envs, linear 150 lines x 200 samples at 0.5 mm (200 x 150 image,
    App. C.1), on the 256^3 volume."""
    spec = c2_spec()
    lab, hu = make_volume(spec)
    return Workload("paper_replica_linear_200x150_100env", [(spec, lab, hu)],
                    [linear_probe(150, 200, 100.0, 0.5)], np.zeros((B, 2), np.int32),
                    dorsal_poses(spec, B, 2001), seed=0x5EED0004)


def surgery3d_probe() -> Probe:
    """The surgery task's 3-D probe (App. C): 50 x 37 pixels at 2 x 2 mm per
    elevation slice (linear, 37 lines at 2 mm, 50 samples over 100 mm); the
    5 slices 10 mm apart come from the elevation sweep of us_sim_render_3d."""
    return linear_probe(37, 50, 100.0, 2.0)


SURGERY3D_SLICES, SURGERY3D_PITCH_MM = 5, 10.0


def workload_surgery3d(B=128):
    """B environments with the 3-D probe above the 256^3 spine volume
    (volumetric images 50 x 37 x 5; App. C trains with 128 parallel envs)."""
    spec = c2_spec()
    lab, hu = make_volume(spec)
    return Workload(f"surgery3d_50x37x5_{B}env", [(spec, lab, hu)], [surgery3d_probe()],
                    np.zeros((B, 2), np.int32), dorsal_poses(spec, B, 2003, tilt_deg=5.0), seed=0x5EED0006)


# --------------------------------------------------------------------------
# surrogate inputs
# --------------------------------------------------------------------------

def surrogate_init(sizes, fan_in, seed: int) -> np.ndarray:
    """Initial network parameters: He-normal weights N(0, 2 / fan_in),
    zero biases (fan_in 0), segment by segment, seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for n, f in zip(sizes, fan_in):
        out.append(rng.normal(0.0, math.sqrt(2.0 / f), int(n)) if f > 0 else np.zeros(int(n)))
    return np.concatenate(out).astype(np.float32)
