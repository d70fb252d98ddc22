"""GPU parity of the render path (persistent cluster kernel, two-pass
batched path and plain per-environment kernels) against the CPU oracle,
through the C ABI."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2507_01152_gb300 import scene

from simhelp import compare, gpu_sim, render_gpu, render_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()


def _check_all(g, o, probes, envs, which, frame_tol=1e-3):
    bad = {}
    for b in which:
        m = compare(g[b], o[b], probes[int(envs[b][1])], frame_tol)
        if m:
            bad[b] = m
    assert not bad, bad


@pytest.mark.parametrize("path", [0, 1])
def test_single_linear_env_128cube(path):
    """1 env, 128^3 volume at 1 mm, linear 128 x 256 to 80 mm."""
    wl = scene.workload_c1()
    sim = gpu_sim(wl)
    g = render_gpu(sim, wl.envs, wl.poses, wl.seed, 0, path=path)
    o = render_oracle(wl, wl.envs, wl.poses, wl.seed, 0, [0])
    _check_all(g, o, wl.probes, wl.envs, [0])
    assert (g[0]["label"] > 0).mean() > 0.5      # the probe looks into the body


@pytest.fixture(scope="module")
def c2():
    wl = scene.workload_c2(64)
    return wl, gpu_sim(wl)


@pytest.fixture(scope="module")
def c2_oracle(c2):
    wl, _ = c2
    return render_oracle(wl, wl.envs, wl.poses, wl.seed, 5, range(64))


@pytest.mark.parametrize("shape", [(8, 32, 0), (1, 32, 0), (1, 16, 0), (1, 16, 1), (1, 8, 1)])
def test_batched_curvilinear_64env_full(c2, c2_oracle, shape):
    """All 64 envs of the 256^3 curvilinear batch, element by element, in the
    launch configurations the benchmark's autotuner chooses from (cluster
    kernel, two-pass path in two grids and in one persistent grid)."""
    wl, sim = c2
    old = sim.get_tuning()
    try:
        sim.set_tuning(shape[0], shape[1], 1, shape[2])
        g = render_gpu(sim, wl.envs, wl.poses, wl.seed, 5, path=0)
    finally:
        sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"])
    _check_all(g, c2_oracle, wl.probes, wl.envs, range(64))


@pytest.mark.parametrize("shape", [(8, 32, 0), (1, 8, 0), (1, 32, 0), (1, 16, 1), (1, 32, 1)])
def test_batched_paths_equal_plain_bitwise(c2, shape):
    """Frames and every intermediate export (labels, voxel indices, envelope,
    log image) of the cluster kernel and of the two-pass path (two grids or
    one persistent grid) equal those of the plain per-environment kernels
    bit for bit."""
    wl, sim = c2
    envs, poses = wl.envs[:12], wl.poses[:12]
    old = sim.get_tuning()
    try:
        sim.set_tuning(shape[0], shape[1], 0, shape[2])
        a = render_gpu(sim, envs, poses, 11, 2, path=0)
    finally:
        sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"])
    b = render_gpu(sim, envs, poses, 11, 2, path=1)
    for x, y in zip(a, b):
        for k in x:
            assert np.array_equal(x[k], y[k]), k


def test_deterministic_and_step_keyed(c2):
    wl, sim = c2
    envs, poses = wl.envs[:6], wl.poses[:6]
    a = render_gpu(sim, envs, poses, 3, 1, debug=False)
    b = render_gpu(sim, envs, poses, 3, 1, debug=False)
    c = render_gpu(sim, envs, poses, 3, 2, debug=False)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x["frame"], y["frame"])
        assert not np.array_equal(x["frame"], z["frame"])   # fresh speckle every step


def test_launch_shape_that_cannot_fit_is_rejected(c2):
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_UNSUPPORTED, US_ERR_INVALID_ARG
    wl, sim = c2
    with pytest.raises(UsError) as e:
        sim.set_tuning(4, 32)          # 64 lines x 512 samples per CTA: too large
    assert e.value.status == US_ERR_UNSUPPORTED
    with pytest.raises(UsError) as e:
        sim.set_tuning(2, 32)          # not a compiled shape
    assert e.value.status == US_ERR_INVALID_ARG
    with pytest.raises(UsError) as e:
        sim.set_tuning(8, 32, 1, 1)    # the persistent grid is a two-pass form
    assert e.value.status == US_ERR_INVALID_ARG


@pytest.mark.parametrize("cs,nw", [(8, 8), (8, 16), (8, 32), (16, 8), (16, 16), (16, 32), (1, 8), (1, 16), (1, 32)])
def test_launch_shapes_agree(c2, cs, nw):
    wl, sim = c2
    envs, poses = wl.envs[:10], wl.poses[:10]
    ref = render_gpu(sim, envs, poses, 21, 0, path=1, debug=False)
    old = sim.get_tuning()
    try:
        for graph in (0, 1):
            for pers in ((0, 1) if cs == 1 else (0,)):
                sim.set_tuning(cs, nw, graph, pers)
                got = render_gpu(sim, envs, poses, 21, 0, path=0, debug=False)
                for x, y in zip(ref, got):
                    assert np.array_equal(x["frame"], y["frame"])
    finally:
        sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"])


def test_graph_replay_updates_arguments(c2):
    """Replays of the captured graph take each call's poses, seed, step and
    frame buffer; the result equals a direct launch every time."""
    wl, sim = c2
    envs = wl.envs[:8]
    off = sim.frame_layout(envs)
    st = torch.cuda.Stream()
    outs = {}
    for graph in (0, 1):
        sim.set_tuning(8, 32, graph)
        for k in range(4):
            P = torch.from_numpy(wl.poses[8 * k:8 * k + 8]).cuda()
            fr = torch.empty(int(off[-1]), device="cuda")
            sim.render(envs, P, 100 + k, k, fr, stream=st)
            st.synchronize()
            outs[(graph, k)] = fr.cpu().numpy()
    sim.set_tuning(8, 32, 1)
    for k in range(4):
        assert np.array_equal(outs[(0, k)], outs[(1, k)])
    assert not np.array_equal(outs[(1, 0)], outs[(1, 1)])


def test_autotune_picks_a_shape_and_caches_it(c2, tmp_path):
    wl, sim = c2
    envs, poses = wl.envs[:16], wl.poses[:16]
    ref = render_gpu(sim, envs, poses, 5, 5, path=1, debug=False)
    P = torch.from_numpy(poses).cuda()
    off = sim.frame_layout(envs)
    fr = torch.empty(int(off[-1]), device="cuda")
    cache = tmp_path / "tune.txt"
    sim.autotune(envs, P, fr, str(cache))
    t1 = sim.get_tuning()
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and f"cs={t1['cluster_size']} nw={t1['warps_per_cta']}" in lines[0]
    assert f"pg={t1['persistent']} wl={t1['wedge_lines']}" in lines[0]
    # a cache line written before the pass-B tile width was a field reads as the widest tile
    old_line = lines[0].split(" wl=")[0] + " ms=0.1\n"
    cache2 = tmp_path / "tune_old.txt"
    cache2.write_text(old_line)
    sim.set_tuning(16, 16)
    sim.autotune(envs, P, fr, str(cache2))
    t2 = sim.get_tuning()
    assert (t2["cluster_size"], t2["warps_per_cta"], t2["persistent"], t2["wedge_lines"]) == \
        (t1["cluster_size"], t1["warps_per_cta"], t1["persistent"], 0)
    assert len(cache2.read_text().splitlines()) == 1
    sim.set_tuning(16, 16)
    sim.autotune(envs, P, fr, str(cache))          # read back from the cache, no new entry
    assert sim.get_tuning() == t1 and len(cache.read_text().splitlines()) == 1
    got = render_gpu(sim, envs, poses, 5, 5, path=0, debug=False)
    for x, y in zip(ref, got):
        assert np.array_equal(x["frame"], y["frame"])
    sim.set_tuning(8, 32, 1)


def _tiny_volume(seed, shape=(14, 16, 18)):
    rng = np.random.default_rng(seed)
    lab = np.repeat(rng.integers(0, 5, (shape[0], shape[1], (shape[2] + 2) // 3)), 3, axis=2)[:, :, :shape[2]]
    hu = rng.integers(-300, 900, shape).astype(np.int16)
    return np.ascontiguousarray(lab.astype(np.uint8)), hu


def _rand_pose(rng, centre):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    t = np.asarray(centre) + rng.uniform(-3, 3, 3)
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


@pytest.mark.parametrize("opt", [scene.Options(1, 1, 0, 1), scene.Options(2, 0, 1, 1), scene.Options(1, 1, 1, 0),
                                 scene.Options(2, 1, 0, 0)])
def test_tiny_random_cases_vs_oracle_and_brute_force(opt):
    """Tiny volumes, ragged probes (line and sample counts that fill no
    tile evenly), random rotations; GPU against the oracle and, for a few,
    against the brute force."""
    lab, hu = _tiny_volume(3)
    spec = scene.VolumeSpec(18, 16, 14, 1.0, 0, 0)
    probes = [scene.linear_probe(7, 37, 9.0, 0.8, psf_sigma_ax_mm=0.5, psf_sigma_lat_mm=1.0),
              scene.curvilinear_probe(9, 70, 8.0, 50.0, 6.0, 13, 11, psf_sigma_ax_mm=0.3, psf_sigma_lat_mm=0.6),
              scene.curvilinear_probe(33, 130, 12.0, 70.0, 5.0, 24, 20, psf_sigma_ax_mm=0.4, psf_sigma_lat_mm=0.5)]
    rng = np.random.default_rng(17)
    B = 24
    envs = np.stack([np.zeros(B), np.arange(B) % 3], axis=1).astype(np.int32)
    poses = np.stack([_rand_pose(rng, (9.0, 8.0, 2.0)) for _ in range(B)])
    wl = scene.Workload("tiny", [(spec, lab, hu)], probes, envs, poses, options=opt, seed=99)
    sim = gpu_sim(wl)
    o = render_oracle(wl, envs, poses, 0xABCDEF0123, 9, range(B))
    for path, shape in ((0, (8, 32, 0)), (0, (1, 8, 0)), (0, (1, 32, 0)), (0, (1, 16, 1)), (1, None)):
        if shape:
            sim.set_tuning(shape[0], shape[1], 0, shape[2])
        g = render_gpu(sim, envs, poses, 0xABCDEF0123, 9, path=path)
        _check_all(g, o, probes, envs, range(B))
    for b in range(3):
        br = brute.render(lab, hu, 1.0, scene.tissue_table(), probes[envs[b][1]], opt, poses[b], env=b,
                          seed=0xABCDEF0123, step=9)
        assert not compare(g[b], br, probes[envs[b][1]])


def test_paper_size_linear_200x150():
    """100 envs, linear 150 lines x 200 samples (200 x 150 image at 0.5 mm)."""
    wl = scene.workload_paper_replica(100)
    sim = gpu_sim(wl)
    g = render_gpu(sim, wl.envs, wl.poses, wl.seed, 0)
    o = render_oracle(wl, wl.envs, wl.poses, wl.seed, 0, range(0, 100, 7))
    _check_all(g, o, wl.probes, wl.envs, range(0, 100, 7))


@pytest.mark.slow
def test_uneven_batch_512env_sampled():
    """512 envs over four 512 x 512 x 256 volumes and three probe types, in
    the fused launch; a sample of envs of every probe type and volume
    checked element by element."""
    wl = scene.workload_c3(512, steps=2)
    sim = gpu_sim(wl)
    poses = wl.poses[1]
    which = list(range(0, 512, 23)) + [511]
    o = render_oracle(wl, wl.envs, poses, wl.seed, 1, which)
    for shape in ((8, 32, 0), (1, 32, 0), (1, 16, 1)):
        sim.set_tuning(shape[0], shape[1], 1, shape[2])
        g = render_gpu(sim, wl.envs, poses, wl.seed, 1)
        _check_all(g, o, wl.probes, wl.envs, which)


def test_host_buffers_match_device(c2):
    wl, sim = c2
    envs, poses = wl.envs[:5], wl.poses[:5]
    ref = render_gpu(sim, envs, poses, 8, 8, debug=False)
    off = sim.frame_layout(envs)
    host = np.zeros(int(off[-1]), np.float32)
    sim.render_host(envs, poses, 8, 8, host)
    for b in range(5):
        assert np.array_equal(host[off[b]:off[b + 1]][:256 * 256].reshape(256, 256), ref[b]["frame"])


def test_empty_batch_and_bad_arguments(c2):
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_INVALID_ARG
    wl, sim = c2
    frames = torch.zeros(256 * 256 * 2, device="cuda")
    sim.render(np.zeros((0, 2), np.int32), torch.zeros((0, 3, 4), device="cuda"), 1, 1, frames)
    P = torch.from_numpy(wl.poses[:2]).cuda()
    with pytest.raises(UsError) as e:
        sim.render(np.array([[0, 5], [0, 0]], np.int32), P, 1, 1, frames)
    assert e.value.status == US_ERR_INVALID_ARG
    with pytest.raises(UsError):
        sim.render(np.array([[1, 0], [0, 0]], np.int32), P, 1, 1, frames)
    with pytest.raises(UsError):
        sim.render(wl.envs[:2], P, 1, 1, frames[1:])          # misaligned frames
    with pytest.raises(UsError):
        sim.render_host(wl.envs[:1], np.full((1, 3, 4), np.nan, np.float32), 1, 1, np.zeros(65536, np.float32))


def test_non_finite_pose_renders_water_and_is_reported(c2):
    from paper_2507_01152_gb300.ussim import UsError
    wl, sim = c2
    poses = wl.poses[:3].copy()
    poses[1, 0, 3] = np.nan
    g = render_gpu(sim, wl.envs[:3], poses, 1, 1, debug=False)
    with pytest.raises(UsError):
        sim.check()
    sim.check()                                   # the error word was cleared
    assert np.all(g[1]["frame"] == 0.0)
    assert np.any(g[0]["frame"] > 0.0)


def test_label_outside_table_rejected_at_create():
    from paper_2507_01152_gb300.ussim import Sim, UsError
    lab = torch.full((4, 4, 4), 9, dtype=torch.uint8, device="cuda")
    hu = torch.zeros((4, 4, 4), dtype=torch.int16, device="cuda")
    with pytest.raises(UsError):
        Sim([(lab, hu, 1.0)], scene.tissue_table(), [scene.linear_probe(8, 16, 8.0, 0.5)])


def test_probe_outside_volume_is_water():
    spec = scene.VolumeSpec(8, 8, 8, 1.0, 0, 0)
    lab = np.full((8, 8, 8), 3, np.uint8)
    hu = np.full((8, 8, 8), 50, np.int16)
    probes = [scene.linear_probe(8, 16, 8.0, 0.5)]
    pose = np.array([[1, 0, 0, 500.0], [0, 1, 0, 500.0], [0, 0, 1, 500.0]], np.float32)[None]
    wl = scene.Workload("far", [(spec, lab, hu)], probes, np.zeros((1, 2), np.int32), pose)
    g = render_gpu(gpu_sim(wl), wl.envs, pose, 1, 1)
    assert np.all(g[0]["nn_index"] == -1) and np.all(g[0]["label"] == 0) and np.all(g[0]["frame"] == 0)


def test_philox_matches_curand(tmp_path):
    """The oracle's Philox (which the speckle parity ties to the CUDA path)
    against NVIDIA's curand_Philox4x32_10 on the device."""
    import ctypes
    import subprocess
    src = tmp_path / "p.cu"
    src.write_text(r'''
#include <curand_kernel.h>
__global__ void k(const uint4* c, const uint2* key, uint4* o, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = curand_Philox4x32_10(c[i], key[i]);
}
extern "C" int run(const unsigned* c, const unsigned* key, unsigned* o, int n) {
  uint4 *dc, *dout; uint2* dk;
  cudaMalloc(&dc, n * 16); cudaMalloc(&dk, n * 8); cudaMalloc(&dout, n * 16);
  cudaMemcpy(dc, c, n * 16, cudaMemcpyHostToDevice); cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice);
  k<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
  int e = (int)cudaMemcpy(o, dout, n * 16, cudaMemcpyDeviceToHost);
  cudaFree(dc); cudaFree(dk); cudaFree(dout);
  return e;
}''')
    so = tmp_path / "p.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC",
                    str(src), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    rng = np.random.default_rng(1)
    n = 4096
    c = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    c[0] = 0
    k[0] = 0
    out = np.zeros((n, 4), np.uint32)
    assert lib.run(c.ctypes.data, k.ctypes.data, out.ctypes.data, n) == 0
    for i in range(0, n, 7):
        assert list(oracle.philox4x32_10(c[i], k[i])) == list(out[i])
    assert list(out[0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]


def test_3d_probe_sweep_equals_2d_renders_and_oracle():
    """The 3-D probe (50 x 37 x 5 at 2 x 2 x 10 mm): each volumetric image,
    in every batched form, equals the plain 2-D renders of its five swept
    planes (host float32 sweep, bit for bit), and sampled slices match the
    oracle."""
    wl = scene.workload_surgery3d(12)
    sim = gpu_sim(wl)
    E, pitch = scene.SURGERY3D_SLICES, scene.SURGERY3D_PITCH_MM
    envs_x = np.repeat(wl.envs, E, axis=0)
    off = sim.frame_layout(envs_x)
    P = torch.from_numpy(np.ascontiguousarray(wl.poses, np.float32)).cuda()
    swept = oracle.sweep_elevation(wl.poses, E, pitch)
    ref = render_gpu(sim, envs_x, swept, wl.seed, 2, path=1, debug=False)
    for shape in ((1, 16, 0), (1, 8, 1), (8, 16, 0)):     # two grids, persistent grid, cluster kernel
        sim.set_tuning(shape[0], shape[1], 1, shape[2])
        fr3 = torch.full((int(off[-1]),), -7.0, device="cuda")
        sim.render_3d(wl.envs, P, E, pitch, wl.seed, 2, fr3)
        torch.cuda.synchronize()
        got = fr3.cpu().numpy()
        for i in range(len(envs_x)):
            assert np.array_equal(got[off[i]:off[i] + 37 * 50].reshape(50, 37), ref[i]["frame"]), (shape, i)
    which = [0, 7, 31, 59]
    o = render_oracle(dataclasses.replace(wl, envs=envs_x, poses=swept), envs_x, swept, wl.seed, 2, which)
    g = render_gpu(sim, envs_x, swept, wl.seed, 2)
    _check_all(g, o, wl.probes, envs_x, which)
    assert np.abs(swept[1, :, 3] - swept[0, :, 3]).sum() > 9.0       # slices 10 mm apart


def test_maximum_probe_sizes_and_widest_psf():
    """Probes of the maximum size (1024 lines x 1024 samples, 1024 x 1024
    output) render through the batched path, bit-identical to the plain
    kernels and within the parity bar of the oracle; so does a maximum-size
    probe with a 48-line lateral PSF reach on either side (pass B stages
    its rows in sample chunks, so every valid probe has a batched shape)."""
    spec = scene.c1_spec()
    lab, hu = scene.make_volume(spec)
    probes = [scene.linear_probe(1024, 1024, 100.0, 0.25),
              scene.curvilinear_probe(1024, 1024, 80.0, 60.0, 40.0, 1024, 1024, psf_sigma_lat_mm=0.2)]
    envs = np.array([[0, 0], [0, 1]], np.int32)
    poses = scene.dorsal_poses(spec, 2, 99)
    wl = scene.Workload("max", [(spec, lab, hu)], probes, envs, poses, seed=11)
    sim = gpu_sim(wl)
    g = render_gpu(sim, envs, poses, wl.seed, 0, path=0)
    p = render_gpu(sim, envs, poses, wl.seed, 0, path=1)
    for x, y in zip(g, p):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    o = render_oracle(wl, envs, poses, wl.seed, 0, [0, 1])
    _check_all(g, o, probes, envs, [0, 1])
    wide = [scene.linear_probe(1024, 1024, 100.0, 0.1, psf_sigma_lat_mm=1.6)]
    wl2 = scene.Workload("wide", [(spec, lab, hu)], wide, envs[:1] * 0, poses[:1], seed=12)
    sim2 = gpu_sim(wl2)
    assert sim2.get_tuning()["cluster_size"] == 1          # two-pass shape found
    gw = render_gpu(sim2, wl2.envs, poses[:1], 12, 0, path=0)
    q = render_gpu(sim2, wl2.envs, poses[:1], 12, 0, path=1)
    for k in q[0]:
        assert np.array_equal(gw[0][k], q[0][k]), k
    o2 = render_oracle(wl2, wl2.envs, poses[:1], 12, 0, [0])
    _check_all(q, o2, wide, wl2.envs, [0])


def test_persistent_grid_wait_runs_out_and_reports(c2):
    """The persistent grid's bounded wait, made to run out: with no pass-A
    group published (the self-test starts the unit counter past them), every
    pass-B tile gives up after its bound, leaves the frames untouched and
    sets the error word; us_sim_check reports US_ERR_TIMEOUT, and the same
    handle then renders normally."""
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_TIMEOUT
    wl, sim = c2
    envs, poses = wl.envs[:8], wl.poses[:8]
    off = sim.frame_layout(envs)
    P = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    frames = torch.full((int(off[-1]),), -7.0, device="cuda")
    old = sim.get_tuning()
    try:
        sim.set_tuning(1, 16, 0, 1)
        sim.selftest_tile_wait(envs, P, frames, 2_000_000)      # ~1 ms per wait
        with pytest.raises(UsError) as e:
            sim.check()
        assert e.value.status == US_ERR_TIMEOUT
        assert bool((frames == -7.0).all())
        sim.check()                                              # the word was cleared
        got = render_gpu(sim, envs, poses, 5, 1, debug=False)
        sim.check()
    finally:
        sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"])
    ref = render_gpu(sim, envs, poses, 5, 1, path=1, debug=False)
    for x, y in zip(ref, got):
        assert np.array_equal(x["frame"], y["frame"])


@pytest.mark.parametrize("B", [1, 2, 3])
def test_persistent_grid_on_tiny_mixed_batches(B):
    """The persistent grid with fewer work units than resident blocks and
    probes of different geometry in one batch (tiles waiting on groups of
    ragged line counts): bit-identical to the plain kernels, both tunings of
    the group size, with and without graph replay."""
    lab, hu = _tiny_volume(5)
    spec = scene.VolumeSpec(18, 16, 14, 1.0, 0, 0)
    probes = [scene.curvilinear_probe(33, 130, 12.0, 70.0, 5.0, 24, 20, psf_sigma_ax_mm=0.4, psf_sigma_lat_mm=0.5),
              scene.linear_probe(7, 37, 9.0, 0.8, psf_sigma_ax_mm=0.5, psf_sigma_lat_mm=1.0)]
    rng = np.random.default_rng(40 + B)
    envs = np.stack([np.zeros(B), np.arange(B) % 2], axis=1).astype(np.int32)
    poses = np.stack([_rand_pose(rng, (9.0, 8.0, 2.0)) for _ in range(B)])
    wl = scene.Workload("tinyp", [(spec, lab, hu)], probes, envs, poses, seed=5)
    sim = gpu_sim(wl)
    ref = render_gpu(sim, envs, poses, 5, 3, path=1)
    for nw in (8, 16, 32):
        for graph in (0, 1):
            sim.set_tuning(1, nw, graph, 1)
            got = render_gpu(sim, envs, poses, 5, 3, path=0) if graph == 0 else \
                render_gpu(sim, envs, poses, 5, 3, path=0, debug=False)
            for x, y in zip(ref, got):
                for k in y:
                    assert np.array_equal(x[k], y[k]), (nw, graph, k)
    sim.check()
    sim.close()


def test_render_timed_reports_each_form_and_renders_the_same(c2):
    """us_sim_render_timed: two durations for the two grids, one for the
    persistent grid and for the cluster kernel; the frames equal
    us_sim_render's."""
    wl, sim = c2
    envs, poses = wl.envs[:8], wl.poses[:8]
    off = sim.frame_layout(envs)
    P = torch.from_numpy(np.ascontiguousarray(poses, np.float32)).cuda()
    old = sim.get_tuning()
    try:
        for shape, n in (((1, 16, 0), 2), ((1, 16, 1), 1), ((8, 32, 0), 1)):
            sim.set_tuning(shape[0], shape[1], 0, shape[2])
            a = torch.full((int(off[-1]),), -7.0, device="cuda")
            b = torch.full((int(off[-1]),), -7.0, device="cuda")
            ms = sim.render_timed(envs, P, 3, 4, a)
            sim.render(envs, P, 3, 4, b)
            torch.cuda.synchronize()
            assert len(ms) == n and all(t > 0 for t in ms), (shape, ms)
            assert torch.equal(a, b), shape
            sim.check()
    finally:
        sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"])


@pytest.mark.parametrize("shape", [(8, 32, 1, 0), (1, 16, 1, 0), (1, 16, 0, 1), (1, 32, 1, 1)])
def test_same_signature_on_two_streams_overlaps_safely(c2, shape):
    """A batch signature's workspace (work lists, line buffer, persistent
    grid counters, cluster work counter, captured graph) is kept per stream:
    renders of one signature queued on two streams with no ordering between
    them give the frames each gives alone."""
    wl, sim = c2
    envs = wl.envs[:16]
    off = sim.frame_layout(envs)
    n = int(off[-1])
    old = sim.get_tuning()
    try:
        sim.set_tuning(*shape)
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        P = [torch.from_numpy(wl.poses[16 * k:16 * k + 16]).cuda() for k in range(2)]
        alone = []
        for k in range(2):
            fr = torch.empty(n, device="cuda")
            sim.render(envs, P[k], 40 + k, k, fr, stream=streams[k])
            streams[k].synchronize()
            alone.append(fr.cpu().numpy())
        for _ in range(3):
            outs = [torch.full((n,), -1.0, device="cuda") for _ in range(2)]
            torch.cuda.synchronize()
            for k in range(2):
                sim.render(envs, P[k], 40 + k, k, outs[k], stream=streams[k])
            torch.cuda.synchronize()
            for k in range(2):
                assert np.array_equal(outs[k].cpu().numpy(), alone[k])
    finally:
        sim.set_tuning(old["cluster_size"], old["warps_per_cta"], old["use_graph"], old.get("persistent", 0))


@pytest.mark.parametrize("nw,pers", [(16, 0), (8, 0), (16, 1)])
def test_pass_b_wedge_widths_agree(nw, pers):
    """Pass-B tiles of 8, 16 or 32 lines (us_tuning.wedge_lines) give the
    frames of the plain per-environment kernels bit for bit, on a batch that
    mixes a linear and two curvilinear probes; a width outside {0, 8, 16,
    32}, or one given to the cluster path, is refused."""
    from paper_2507_01152_gb300.ussim import UsError, US_ERR_INVALID_ARG
    spec = scene.VolumeSpec(128, 128, 128, 1.0, 2, 77)
    lab, hu = scene.make_volume(spec)
    probes = [scene.linear_probe(64, 128, 80.0, 0.5), scene.curvilinear_probe(96, 192, 80.0, 60.0, 40.0, 96, 96),
              scene.curvilinear_probe(128, 256, 80.0, 60.0, 40.0, 128, 128)]
    envs = np.array([[0, b % 3] for b in range(9)], np.int32)
    wl = scene.Workload("mix", [(spec, lab, hu)], probes, envs, scene.dorsal_poses(spec, 9, 12), seed=3)
    sim = gpu_sim(wl)
    ref = render_gpu(sim, wl.envs, wl.poses, 8, 1, path=1, debug=False)
    for wedge in (8, 16, 32, 0):
        sim.set_tuning(1, nw, 1, pers, wedge)
        assert sim.get_tuning()["wedge_lines"] == wedge
        for step in range(2):      # the second call replays the graph captured for this width
            got = render_gpu(sim, wl.envs, wl.poses, 8, 1, path=0, debug=False)
            for x, y in zip(ref, got):
                assert np.array_equal(x["frame"], y["frame"]), (wedge, step)
    for bad in ((1, 16, 1, 0, 12), (8, 32, 1, 0, 16)):
        with pytest.raises(UsError) as e:
            sim.set_tuning(*bad)
        assert e.value.status == US_ERR_INVALID_ARG
    sim.close()


def test_host_render_in_sub_batches_matches_device(c2):
    """A batch whose frames pass 16 MB goes to the host in sub-batches (each
    copied while the next renders): the frames equal a device render of the
    whole batch bit for bit, into pinned and into pageable host memory."""
    wl, sim = c2
    B = 170                                    # 170 x 256 KB of frames: four sub-batches
    envs = np.zeros((B, 2), np.int32)
    poses = np.ascontiguousarray(np.stack([wl.poses[b % 64] for b in range(B)]), np.float32)
    off = sim.frame_layout(envs)
    assert int(off[-1]) * 4 > 40 * 2 ** 20
    P = torch.from_numpy(poses).cuda()
    dev = torch.empty(int(off[-1]), device="cuda")
    sim.render(envs, P, 9, 4, dev)
    torch.cuda.synchronize()
    want = dev.cpu().numpy()
    for pinned in (True, False):
        host = torch.full((int(off[-1]),), -3.0).pin_memory() if pinned else torch.full((int(off[-1]),), -3.0)
        sim.render_host(envs, poses, 9, 4, host.numpy())
        assert np.array_equal(host.numpy(), want), pinned


@pytest.mark.parametrize("shape", [(1, 16, 1, 0, 32), (1, 8, 1, 0, 16), (1, 16, 1, 1, 32), (8, 32, 1, 0, 0)])
def test_graph_replays_of_a_mixed_probe_batch_match_plain(shape):
    """Graph capture and replay (an explicit stream) of a batch whose envs
    use three probes of different sizes, so that the two grids launch only
    each env's own work units: every replay, with fresh poses and steps,
    equals the plain per-environment kernels bit for bit."""
    spec = scene.VolumeSpec(128, 128, 128, 1.0, 2, 91)
    lab, hu = scene.make_volume(spec)
    probes = [scene.curvilinear_probe(128, 256, 80.0, 60.0, 40.0, 128, 128),
              scene.curvilinear_probe(96, 192, 80.0, 60.0, 40.0, 96, 96), scene.linear_probe(64, 128, 80.0, 0.5)]
    B = 24
    envs = np.array([[0, (b * 7) % 3] for b in range(B)], np.int32)
    poses = scene.dorsal_poses(spec, 3 * B, 13).reshape(3, B, 3, 4)
    wl = scene.Workload("mix3", [(spec, lab, hu)], probes, envs, poses[0], seed=4)
    sim = gpu_sim(wl)
    sim.set_tuning(*shape)
    st = torch.cuda.Stream()
    off = sim.frame_layout(envs)
    n = int(off[-1])
    for k in range(3):
        P = torch.from_numpy(np.ascontiguousarray(poses[k])).cuda()
        got = torch.full((n,), -7.0, device="cuda")
        sim.render(envs, P, 17, k, got, stream=st)
        st.synchronize()
        want = torch.full((n,), -7.0, device="cuda")
        sim.render_plain(envs, P, 17, k, want, stream=st)
        st.synchronize()
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy()), (shape, k)
    sim.close()


def test_host_render_in_sub_batches_with_mixed_frame_sizes():
    """Sub-batched host renders of a batch mixing three frame sizes (the
    sub-batch boundaries fall between envs of different probes): equal to
    the device render of the whole batch."""
    spec = scene.VolumeSpec(128, 128, 128, 1.0, 2, 93)
    lab, hu = scene.make_volume(spec)
    probes = [scene.curvilinear_probe(128, 256, 80.0, 60.0, 40.0, 128, 128),
              scene.curvilinear_probe(96, 192, 80.0, 60.0, 40.0, 96, 96), scene.linear_probe(64, 128, 80.0, 0.5)]
    B = 420
    envs = np.array([[0, (b * 5) % 3] for b in range(B)], np.int32)
    poses = np.ascontiguousarray(scene.dorsal_poses(spec, B, 17), np.float32)
    wl = scene.Workload("mix3h", [(spec, lab, hu)], probes, envs, poses, seed=6)
    sim = gpu_sim(wl)
    off = sim.frame_layout(envs)
    assert int(off[-1]) * 4 >= 16 * 2 ** 20       # sub-batched
    dev = torch.empty(int(off[-1]), device="cuda")
    sim.render(envs, torch.from_numpy(poses).cuda(), 3, 9, dev)
    torch.cuda.synchronize()
    host = torch.full((int(off[-1]),), -3.0).pin_memory()
    sim.render_host(envs, poses, 3, 9, host.numpy())
    assert np.array_equal(host.numpy(), dev.cpu().numpy())
    sim.close()
