"""Thin ctypes binding of libussim (include/ussim.h).

Argument marshalling only: every step of the render runs in the CUDA
library.  Device buffers are passed as torch CUDA tensors (torch provides
device memory and streams, nothing else); host buffers as numpy arrays.
Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

US_OK, US_ERR_INVALID_ARG, US_ERR_CUDA, US_ERR_OOM, US_ERR_TIMEOUT, US_ERR_UNSUPPORTED, US_ERR_INTERNAL = range(7)


class UsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "US_OK", 1: "US_ERR_INVALID_ARG", 2: "US_ERR_CUDA", 3: "US_ERR_OOM", 4: "US_ERR_TIMEOUT",
           5: "US_ERR_UNSUPPORTED", 6: "US_ERR_INTERNAL"}


class us_volume(C.Structure):
    _fields_ = [("labels", C.c_void_p), ("hu", C.c_void_p), ("nx", C.c_int32), ("ny", C.c_int32),
                ("nz", C.c_int32), ("voxel_mm", C.c_float)]


class us_tissue(C.Structure):
    _fields_ = [("alpha_db_cm_mhz", C.c_float), ("z_mrayl", C.c_float), ("mu0", C.c_float),
                ("sigma0", C.c_float), ("mu1", C.c_float)]


class us_probe(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_lines", C.c_int32), ("n_samples", C.c_int32),
                ("depth_mm", C.c_float), ("pitch_mm", C.c_float), ("fan_deg", C.c_float),
                ("radius_mm", C.c_float), ("out_w", C.c_int32), ("out_h", C.c_int32),
                ("f_mhz", C.c_float), ("e0", C.c_float), ("psf_sigma_ax_mm", C.c_float),
                ("psf_sigma_lat_mm", C.c_float), ("dyn_range_db", C.c_float)]


class us_options(C.Structure):
    _fields_ = [("refl_power", C.c_int32), ("transmission", C.c_int32), ("z_mode", C.c_int32),
                ("speckle", C.c_int32), ("speckle_anchor", C.c_int32), ("speckle_levels", C.c_int32),
                ("speckle_cell_mm", C.c_float), ("volume_layout", C.c_int32)]


class us_env(C.Structure):
    _fields_ = [("volume_id", C.c_int32), ("probe_id", C.c_int32)]


class us_tuning(C.Structure):
    _fields_ = [("cluster_size", C.c_int32), ("warps_per_cta", C.c_int32), ("use_graph", C.c_int32),
                ("persistent", C.c_int32), ("wedge_lines", C.c_int32)]


class us_surr_config(C.Structure):
    _fields_ = [("base_channels", C.c_int32), ("height", C.c_int32), ("width", C.c_int32),
                ("max_batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float)]


# name -> (restype, argtypes) for every entry point of include/*.h
_P = C.c_void_p
_I = C.c_int32
SIGNATURES = {
    "us_sim_create": (C.c_int, [C.POINTER(us_volume), C.c_int32, C.POINTER(us_tissue), C.c_int32,
                                C.POINTER(us_probe), C.c_int32, C.POINTER(us_options), C.POINTER(_P)]),
    "us_sim_destroy": (None, [_P]),
    "us_sim_refresh_volumes": (C.c_int, [_P, _P]),
    "us_sim_set_hu_reference": (C.c_int, [_P, _P, C.c_int32, C.c_float, C.c_float]),
    "us_sim_hist_match": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, _P, _P]),
    "us_sim_selftest_tile_wait": (C.c_int, [_P, _P, C.c_int32, _P, _P, C.c_int64, _P]),
    "us_sim_frame_layout": (C.c_int, [_P, _P, C.c_int32, _P]),
    "us_sim_beam_layout": (C.c_int, [_P, _P, C.c_int32, _P]),
    "us_sim_render": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P]),
    "us_sim_render_plain": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P]),
    "us_sim_render_plain_static": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P]),
    "us_sim_render_debug": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P, _P, _P, _P,
                                      C.c_int32, _P]),
    "us_sim_render_host": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P]),
    "us_sim_check": (C.c_int, [_P, _P]),
    "us_sim_render_timed": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P, _P, _P]),
    "us_sim_render_3d": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int32, C.c_float, C.c_uint64, C.c_uint64, _P, _P]),
    "us_sim_sweep_poses": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_float, _P, _P]),
    "us_sim_recon_words": (C.c_int64, [_P]),
    "us_sim_recon_update": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, C.c_int32, C.c_float, _P, _P,
                                      _P, C.c_int32, _P]),
    "us_sim_recon_observe": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, C.c_int32, _P, _P]),
    "us_sim_sample_slices": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P]),
    "us_sim_sample_slices_grid": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P]),
    "us_sim_resize_frames": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P]),
    "us_sim_render_audit": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P, C.c_float, C.c_float,
                                      _P, _P, _P]),
    "us_sim_render_gated": (C.c_int, [_P, _P, C.c_int32, _P, C.c_uint64, C.c_uint64, _P, _P, C.c_float, _P, _P]),
    "us_sim_get_tuning": (C.c_int, [_P, C.POINTER(us_tuning)]),
    "us_sim_set_tuning": (C.c_int, [_P, C.POINTER(us_tuning)]),
    "us_sim_autotune": (C.c_int, [_P, _P, C.c_int32, _P, _P, C.c_char_p, _P]),
    "us_sim_last_error": (C.c_char_p, [_P]),
    "us_status_string": (C.c_char_p, [C.c_int]),
    "us_gemm_bf16_nt": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P]),
    "us_conv3x3_fwd": (C.c_int, [_P, _I, _I, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _I, _I, _P, _P]),
    "us_conv3x3_dgrad": (C.c_int, [_P, _I, _I, _P, _P, _I, _I, _P, _I, _I, _I, _I, _I, _I, _I, _I, _I, _P, _P]),
    "us_conv3x3_wgrad": (C.c_int, [_P, _I, _I, _P, _I, _I, _P, _I, _I, _I, _I, _I, _I, _P, _P]),
    "us_convT2x2_fwd": (C.c_int, [_P, _I, _I, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _I, _P, _P]),
    "us_convT2x2_dgrad": (C.c_int, [_P, _I, _I, _P, _P, _I, _I, _P, _I, _I, _I, _I, _I, _I, _I, _I, _P, _P]),
    "us_convT2x2_wgrad": (C.c_int, [_P, _I, _I, _P, _I, _I, _P, _I, _I, _I, _I, _I, _P, _P]),
    "us_surr_param_segments": (C.c_int32, [C.POINTER(us_surr_config), C.c_int32, _P, _P, _P]),
    "us_surr_num_params": (C.c_int64, [C.POINTER(us_surr_config)]),
    "us_surr_create": (C.c_int, [C.POINTER(us_surr_config), _P, C.POINTER(_P)]),
    "us_surr_destroy": (None, [_P]),
    "us_surr_last_error": (C.c_char_p, [_P]),
    "us_surr_forward": (C.c_int, [_P, _P, _P, _I, _P]),
    "us_surr_train_step": (C.c_int, [_P, _P, _P, _I, _P, _I, _P]),
    "us_surr_metrics": (C.c_int, [_P, _P, _P, _I, _P, _P]),
    "us_surr_metrics_hw": (C.c_int, [_P, _P, _P, _I, _I, _I, _P, _P]),
    "us_surr_gan_num_params": (C.c_int64, [C.c_int32]),
    "us_surr_gan_enable": (C.c_int, [_P, C.c_int32, _P, C.c_float, C.c_float]),
    "us_surr_gan_disc_step": (C.c_int, [_P, _P, _P, C.c_int32, _P, C.c_int32, _P]),
    "us_surr_gan_get": (C.c_int, [_P, _P, _P]),
    "us_surr_num_features": (C.c_int32, [_P]),
    "us_surr_features": (C.c_int, [_P, C.c_int32, _P, _P]),
    "us_surr_predict_error": (C.c_int, [_P, C.c_int32, _P, _P]),
    "us_surr_fit_error_head": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float]),
    "us_surr_get_params": (C.c_int, [_P, _P]),
    "us_surr_get_grads": (C.c_int, [_P, _P]),
    "us_surr_check": (C.c_int, [_P, _P]),
    "us_surr_save": (C.c_int, [_P, C.c_char_p]),
    "us_surr_load": (C.c_int, [_P, C.c_char_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libussim.so; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"libussim.so not built ({_build.LIB}); run paper_2507_01152_gb300.build")
            _build.build()
        L = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def gemm_bf16_nt(A, B, C, err, stream=None):
    """C = A B^T on the tcgen05 tile kernel (A [M][K], B [N][K] bf16; C fp32)."""
    L = load()
    M, K = A.shape
    N = B.shape[0]
    st = L.us_gemm_bf16_nt(_ptr(A), _ptr(B), _ptr(C), M, N, K, _ptr(err), _stream_handle(stream))
    if st != US_OK:
        raise UsError(st, "us_gemm_bf16_nt")


def op(name, *args, stream=None):
    """Call an operator entry point: tensors -> device pointers, ints as is;
    the trailing stream argument is appended."""
    L = load()
    conv = [(_ptr(a) if not isinstance(a, (int, np.integer)) else int(a)) for a in args]
    st = getattr(L, name)(*conv, _stream_handle(stream))
    if st != US_OK:
        raise UsError(st, name)


def sweep_poses(poses, n_elev, elev_pitch_mm, out, stream=None):
    """The 3-D probe's elevation sweep on the device (us_sim_sweep_poses):
    poses [B][3][4] -> out [B * n_elev][3][4], both device float32."""
    L = load()
    B = int(poses.shape[0])
    st = L.us_sim_sweep_poses(_ptr(poses), B, int(n_elev), float(elev_pitch_mm), _ptr(out), _stream_handle(stream))
    if st != US_OK:
        raise UsError(st, "us_sim_sweep_poses")


def make_probe(p) -> us_probe:
    return us_probe(p.kind, p.n_lines, p.n_samples, p.depth_mm, p.pitch_mm, p.fan_deg, p.radius_mm,
                    p.out_w, p.out_h, p.f_mhz, p.e0, p.psf_sigma_ax_mm, p.psf_sigma_lat_mm, p.dyn_range_db)


def make_envs(envs) -> C.Array:
    """us_env array of (volume_id, probe_id) rows: one buffer copy (us_env
    is two int32, the layout of an int32 [B][2] array)"""
    envs = np.ascontiguousarray(envs, np.int32).reshape(-1, 2)
    if len(envs) == 0:
        return (us_env * 1)()
    return (us_env * len(envs)).from_buffer_copy(envs.tobytes())


class Sim:
    """A simulator handle.  volumes: list of (labels, hu, voxel_mm) with
    labels/hu torch CUDA tensors ([nz][ny][nx] uint8 / int16), kept alive
    here; table: list of tissue records; probes: list of probe records."""

    def __init__(self, volumes, table, probes, options=None):
        L = load()
        self._keep = [(l, h) for (l, h, _) in volumes]
        vols = (us_volume * len(volumes))()
        for i, (lab, hu, vox) in enumerate(volumes):
            nz, ny, nx = lab.shape
            vols[i] = us_volume(_ptr(lab), _ptr(hu), nx, ny, nz, vox)
        tab = (us_tissue * len(table))()
        for i, t in enumerate(table):
            tab[i] = us_tissue(t.alpha_db_cm_mhz, t.z_mrayl, t.mu0, t.sigma0, t.mu1)
        prs = (us_probe * len(probes))(*[make_probe(p) for p in probes])
        opt = None
        if options is not None:
            opt = us_options(options.refl_power, options.transmission, options.z_mode, options.speckle,
                             getattr(options, "speckle_anchor", 0), getattr(options, "speckle_levels", 1),
                             getattr(options, "speckle_cell_mm", 0.25), getattr(options, "volume_layout", 0))
        h = C.c_void_p()
        st = L.us_sim_create(vols, len(volumes), tab, len(table), prs, len(probes),
                             C.byref(opt) if opt is not None else None, C.byref(h))
        if st != US_OK:
            raise UsError(st, "us_sim_create failed")
        self.h = h
        self.probes = list(probes)
        self._lib = L

    # ------------------------------------------------------------ helpers
    def _check(self, st):
        if st != US_OK:
            raise UsError(st, self._lib.us_sim_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.us_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- ABI
    def frame_layout(self, envs) -> np.ndarray:
        e = make_envs(envs)
        B = len(np.asarray(envs).reshape(-1, 2))
        off = np.zeros(B + 1, np.int64)
        self._check(self._lib.us_sim_frame_layout(self.h, e, B, off.ctypes.data))
        return off

    def beam_layout(self, envs) -> np.ndarray:
        e = make_envs(envs)
        B = len(np.asarray(envs).reshape(-1, 2))
        off = np.zeros(B + 1, np.int64)
        self._check(self._lib.us_sim_beam_layout(self.h, e, B, off.ctypes.data))
        return off

    def render(self, envs, poses, seed, step, frames, stream=None, envs_c=None):
        B = poses.shape[0] if poses is not None else 0
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_render(self.h, e, B, _ptr(poses), seed, step, _ptr(frames),
                                            _stream_handle(stream)))

    def render_plain(self, envs, poses, seed, step, frames, stream=None, envs_c=None):
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_render_plain(self.h, e, B, _ptr(poses), seed, step, _ptr(frames),
                                                  _stream_handle(stream)))

    def render_plain_static(self, envs, poses, seed, step, frames, stream=None, envs_c=None):
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_render_plain_static(self.h, e, B, _ptr(poses), seed, step, _ptr(frames),
                                                         _stream_handle(stream)))

    def render_debug(self, envs, poses, seed, step, frames, envelope=None, logimg=None, nn_index=None,
                     label=None, path=0, stream=None):
        B = poses.shape[0]
        self._check(self._lib.us_sim_render_debug(self.h, make_envs(envs), B, _ptr(poses), seed, step,
                                                  _ptr(frames), _ptr(envelope), _ptr(logimg), _ptr(nn_index),
                                                  _ptr(label), path, _stream_handle(stream)))

    def render_host(self, envs, poses_host, seed, step, frames_host, stream=None, envs_c=None):
        poses_host = np.ascontiguousarray(poses_host, np.float32)
        B = poses_host.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_render_host(self.h, e, B, _ptr(poses_host), seed, step, _ptr(frames_host),
                                                 _stream_handle(stream)))

    def render_3d(self, envs, poses, n_elev, elev_pitch_mm, seed, step, frames, stream=None):
        """Volumetric frames of a 3-D probe: each env's plane swept over n_elev
        elevation offsets; frames as frame_layout(np.repeat(envs, n_elev, 0))."""
        B = poses.shape[0]
        self._check(self._lib.us_sim_render_3d(self.h, make_envs(envs), B, _ptr(poses), n_elev,
                                               float(elev_pitch_mm), seed, step, _ptr(frames),
                                               _stream_handle(stream)))

    def recon_words(self):
        return int(self._lib.us_sim_recon_words(self.h))

    def recon_update(self, envs, poses, seed, step, bone_label, p_miss, bitmaps, points, counts, stream=None,
                     envs_c=None):
        """add one frame per env to the reconstructions (bitmaps uint32 [B][recon_words()],
        points int32 [B][cap], counts int32 [B]: device tensors, zeroed to start)"""
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_recon_update(self.h, e, B, _ptr(poses), seed, step, bone_label,
                                                  float(p_miss), _ptr(bitmaps), _ptr(points), _ptr(counts),
                                                  points.shape[1], _stream_handle(stream)))

    def recon_observe(self, envs, poses, points, counts, obs, stream=None, envs_c=None):
        """the reconstructions voxelized in each env's probe frame: obs uint8 [B][40][40][40]"""
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_recon_observe(self.h, e, B, _ptr(poses), _ptr(points),
                                                   _ptr(counts), points.shape[1], _ptr(obs), _stream_handle(stream)))

    def render_timed(self, envs, poses, seed, step, frames, stream=None, envs_c=None):
        """The tuned render with per-kernel CUDA-event times (ms): a list of
        one (cluster kernel) or two (two-pass: pass A, pass B) durations."""
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        ms = (C.c_float * 2)()
        n = C.c_int32(0)
        self._check(self._lib.us_sim_render_timed(self.h, e, B, _ptr(poses), seed, step, _ptr(frames), ms, C.byref(n),
                                                  _stream_handle(stream)))
        return [float(ms[i]) for i in range(n.value)]

    def check(self, stream=None):
        self._check(self._lib.us_sim_check(self.h, _stream_handle(stream)))

    def selftest_tile_wait(self, envs, poses, frames, wait_cycles, stream=None):
        """Run the persistent grid with no pass-A group published, so every
        tile's bounded wait runs out (us_sim_check then reports
        US_ERR_TIMEOUT)."""
        B = poses.shape[0]
        self._check(self._lib.us_sim_selftest_tile_wait(self.h, make_envs(envs), B, _ptr(poses), _ptr(frames),
                                                        int(wait_cycles), _stream_handle(stream)))

    def set_hu_reference(self, ref_cum, h0, bin_width):
        """Reference cumulative bin counts (int64 numpy array) of the CT
        histogram matching, or None to switch it off."""
        if ref_cum is None:
            self._check(self._lib.us_sim_set_hu_reference(self.h, None, 0, 0.0, 1.0))
            return
        import numpy as np
        r = np.ascontiguousarray(ref_cum, np.int64)
        self._check(self._lib.us_sim_set_hu_reference(self.h, r.ctypes.data, len(r), float(h0), float(bin_width)))

    def hist_match(self, hu, mask, out, stream=None):
        """Histogram matching of hu (float32 CUDA [B][n_pix]) into out;
        mask uint8 CUDA [B][n_pix] or None."""
        B, n = hu.shape
        self._check(self._lib.us_sim_hist_match(self.h, _ptr(hu), _ptr(mask) if mask is not None else None, B, n,
                                                _ptr(out), _stream_handle(stream)))

    def refresh_volumes(self, stream=None):
        """Re-read the volumes after their contents changed (label check,
        corner layout of the HU grid); synchronous."""
        self._check(self._lib.us_sim_refresh_volumes(self.h, _stream_handle(stream)))

    def render_gated(self, envs, poses, seed, step, frames, score, threshold, n_rendered=None, stream=None,
                     envs_c=None):
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_render_gated(self.h, e, B, _ptr(poses), seed, step, _ptr(frames), _ptr(score),
                                                  float(threshold), _ptr(n_rendered), _stream_handle(stream)))

    def render_audit(self, envs, poses, seed, step, audit_frames, score, threshold, fraction, flags=None,
                     n_audited=None, stream=None, envs_c=None):
        """physics render of the seeded audit subset of the frames the gate keeps"""
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_render_audit(self.h, e, B, _ptr(poses), seed, step, _ptr(audit_frames),
                                                  _ptr(score), float(threshold), float(fraction), _ptr(flags),
                                                  _ptr(n_audited), _stream_handle(stream)))

    def sample_slices_grid(self, envs, poses, H, W, out, stream=None, envs_c=None):
        """surrogate input [B][H][W][8] bf16 on an H x W grid over each env's field"""
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_sample_slices_grid(self.h, e, B, _ptr(poses), int(H), int(W), _ptr(out),
                                                        _stream_handle(stream)))

    def resize_frames(self, envs, src, frames, stream=None, envs_c=None):
        """src [B][H][W] float32 -> frames in the batch's frame layout"""
        B, H, W = src.shape
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_resize_frames(self.h, e, B, _ptr(src), H, W, _ptr(frames),
                                                   _stream_handle(stream)))

    def sample_slices(self, envs, poses, out, stream=None, envs_c=None):
        """surrogate input [B][H][W][8] bf16 (out: torch bfloat16 CUDA tensor)"""
        B = poses.shape[0]
        e = envs_c if envs_c is not None else make_envs(envs)
        self._check(self._lib.us_sim_sample_slices(self.h, e, B, _ptr(poses), _ptr(out), _stream_handle(stream)))

    def get_tuning(self) -> dict:
        t = us_tuning()
        self._check(self._lib.us_sim_get_tuning(self.h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in us_tuning._fields_}

    def set_tuning(self, cluster_size, warps_per_cta, use_graph=None, persistent=0, wedge_lines=0):
        if use_graph is None:
            use_graph = self.get_tuning()["use_graph"]
        t = us_tuning(cluster_size, warps_per_cta, use_graph, persistent, wedge_lines)
        self._check(self._lib.us_sim_set_tuning(self.h, C.byref(t)))

    def autotune(self, envs, poses, frames, cache_path=None, stream=None):
        B = poses.shape[0]
        self._check(self._lib.us_sim_autotune(self.h, make_envs(envs), B, _ptr(poses), _ptr(frames),
                                              cache_path.encode() if cache_path else None,
                                              _stream_handle(stream)))


class Surrogate:
    """Handle of the learned surrogate (include/ussim_surrogate.h)."""

    def __init__(self, base_channels, height, width, max_batch, init_params, lr=2e-4, beta1=0.9, beta2=0.999,
                 eps=1e-8):
        L = load()
        self.cfg = us_surr_config(base_channels, height, width, max_batch, lr, beta1, beta2, eps)
        n = L.us_surr_num_params(C.byref(self.cfg))
        init = np.ascontiguousarray(init_params, np.float32)
        if n < 0 or init.size != n:
            raise UsError(US_ERR_INVALID_ARG, f"expected {n} parameters, got {init.size}")
        h = C.c_void_p()
        st = L.us_surr_create(C.byref(self.cfg), init.ctypes.data, C.byref(h))
        if st != US_OK:
            raise UsError(st, "us_surr_create")
        self.h, self.n_params, self._lib = h, n, L

    @staticmethod
    def segments(base_channels, height=256, width=256):
        """(offsets, sizes, fan_in) of the parameter segments"""
        L = load()
        cfg = us_surr_config(base_channels, height, width, 1, 1e-3, 0.9, 0.999, 1e-8)
        n = L.us_surr_param_segments(C.byref(cfg), 0, None, None, None)
        off, size, fan = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int32)
        L.us_surr_param_segments(C.byref(cfg), n, off.ctypes.data, size.ctypes.data, fan.ctypes.data)
        return off, size, fan

    @staticmethod
    def num_params(base_channels, height=256, width=256):
        cfg = us_surr_config(base_channels, height, width, 1, 1e-3, 0.9, 0.999, 1e-8)
        return load().us_surr_num_params(C.byref(cfg))

    def _check(self, st):
        if st != US_OK:
            raise UsError(st, self._lib.us_surr_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.us_surr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, x, y, stream=None):
        self._check(self._lib.us_surr_forward(self.h, _ptr(x), _ptr(y), x.shape[0], _stream_handle(stream)))

    def train_step(self, x, target, loss_out, update=True, stream=None):
        self._check(self._lib.us_surr_train_step(self.h, _ptr(x), _ptr(target), x.shape[0], _ptr(loss_out),
                                                 1 if update else 0, _stream_handle(stream)))

    def metrics(self, pred, target, out, stream=None):
        self._check(self._lib.us_surr_metrics(self.h, _ptr(pred), _ptr(target), pred.shape[0], _ptr(out),
                                              _stream_handle(stream)))

    def gan_enable(self, cd, init, gan_weight=0.01, lr=2e-4):
        """enable the GAN term with a discriminator of width cd (init: host float32 parameters)"""
        init = np.ascontiguousarray(init, np.float32)
        n = int(self._lib.us_surr_gan_num_params(int(cd)))
        if init.size != n:
            raise ValueError(f"discriminator of width {cd} has {n} parameters, got {init.size}")
        self._gan_n = n
        self._check(self._lib.us_surr_gan_enable(self.h, int(cd), _ptr(init), float(gan_weight), float(lr)))

    def gan_disc_step(self, x, real, loss_out, update=True, stream=None):
        self._check(self._lib.us_surr_gan_disc_step(self.h, _ptr(x), _ptr(real), x.shape[0], _ptr(loss_out),
                                                    1 if update else 0, _stream_handle(stream)))

    def gan_params_grads(self):
        p = np.zeros(self._gan_n, np.float32)
        g = np.zeros(self._gan_n, np.float32)
        self._check(self._lib.us_surr_gan_get(self.h, _ptr(p), _ptr(g)))
        return p, g

    def metrics_hw(self, pred, target, out, stream=None):
        """per-frame L1 / SSIM of [B][H][W] frames of any size up to the network's"""
        B, H, W = pred.shape
        self._check(self._lib.us_surr_metrics_hw(self.h, _ptr(pred), _ptr(target), B, H, W, _ptr(out),
                                                 _stream_handle(stream)))

    def num_features(self):
        return self._lib.us_surr_num_features(self.h)

    def features(self, B, out, stream=None):
        self._check(self._lib.us_surr_features(self.h, B, _ptr(out), _stream_handle(stream)))

    def predict_error(self, B, out, stream=None):
        self._check(self._lib.us_surr_predict_error(self.h, B, _ptr(out), _stream_handle(stream)))

    def fit_error_head(self, feat, target, ridge=1e-3):
        feat = np.ascontiguousarray(feat, np.float32)
        target = np.ascontiguousarray(target, np.float32)
        self._check(self._lib.us_surr_fit_error_head(self.h, feat.ctypes.data, target.ctypes.data, len(target),
                                                     float(ridge)))

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        self._check(self._lib.us_surr_get_params(self.h, out.ctypes.data))
        return out

    def grads(self):
        out = np.zeros(self.n_params, np.float32)
        self._check(self._lib.us_surr_get_grads(self.h, out.ctypes.data))
        return out

    def check(self, stream=None):
        self._check(self._lib.us_surr_check(self.h, _stream_handle(stream)))

    def save(self, path):
        self._check(self._lib.us_surr_save(self.h, path.encode()))

    def load(self, path):
        self._check(self._lib.us_surr_load(self.h, path.encode()))
