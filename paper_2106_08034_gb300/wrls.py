"""Thin ctypes binding of libwrls.so (C ABI in include/wrls.h).

Argument marshalling only: every step of the denoiser runs in the library's CUDA kernels.
Functions keep the C names. Buffers may be torch tensors (their data_ptr() is passed;
device tensors for the device entry points, CPU tensors for wrls_denoise_frame_host) or
raw integer addresses. CUDA streams may be torch.cuda.Stream objects, raw handles or None.

Loading raises if the library has not been built (``__graft_entry__.build()`` or
``python -m paper_2106_08034_gb300.build``): there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwrls.so")

WRLS_OK = 0
WRLS_ERR_INVALID_ARG = 1
WRLS_ERR_OOM = 2
WRLS_ERR_CUDA = 3
WRLS_ERR_STATE = 4
WRLS_ERR_TIMEOUT = 5

WRLS_STATE_F32 = 0
WRLS_STATE_BF16 = 1
WRLS_STATE_F16 = 2

N_STATE = 25

# Every symbol include/wrls.h declares (checked by the ABI test).
EXPORTED = [
    "wrls_params_default", "wrls_state_bytes", "wrls_stream_create", "wrls_stream_set_cuda_stream",
    "wrls_denoise_frame", "wrls_denoise_frame_host", "wrls_stream_reset", "wrls_stream_destroy",
    "wrls_stream_read_state", "wrls_stream_write_state", "wrls_stream_state_stats", "wrls_stream_frames", "wrls_last_error",
    "wrls_stream_enable_timing", "wrls_stream_kernel_times", "wrls_stream_check",
    "wrls_stream_autotune", "wrls_stream_set_blend_config",
    "wrls_stream_set_debug",
    "wrls_batch_create", "wrls_batch_set_cuda_stream", "wrls_batch_tick", "wrls_batch_destroy",
    "wrls_batch_tick_static", "wrls_denoise_sequence", "wrls_denoise_sequence_host", "wrls_stream_set_overlap",
    "wrls_recon_params_default", "wrls_reconstruct", "wrls_velocity_from_world", "wrls_render_vpt",
    "wrls_denoise_batch",
]


class WrlsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("wrls status %d: %s" % (status, message))
        self.status = status


class wrls_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("lambda_", ctypes.c_float), ("h", ctypes.c_float), ("alpha", ctypes.c_float),
        ("eps", ctypes.c_float), ("p0_delta", ctypes.c_float), ("sigma_s", ctypes.c_float),
        ("h_s", ctypes.c_float), ("p_trace_max", ctypes.c_float),
        ("radius", ctypes.c_int32), ("weight_mode", ctypes.c_int32), ("clamp_mode", ctypes.c_int32),
        ("blend_mode", ctypes.c_int32), ("feature_mode", ctypes.c_int32), ("init_mode", ctypes.c_int32),
        ("state_precision", ctypes.c_int32), ("n_features", ctypes.c_int32),
        ("n_gbuf", ctypes.c_int32), ("reproj_filter", ctypes.c_int32),
    ]


class wrls_recon_params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("sigma", ctypes.c_float), ("radius", ctypes.c_float)]


class wrls_vpt_scene(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("seed", ctypes.c_uint32 * 2), ("eye", ctypes.c_float * 3),
                ("inv_view_proj", ctypes.c_float * 16), ("n_blobs", ctypes.c_int32), ("blobs", ctypes.c_float * 80),
                ("mu_max", ctypes.c_float), ("tf_lo", ctypes.c_float), ("tf_hi", ctypes.c_float),
                ("albedo", ctypes.c_float), ("color_lo", ctypes.c_float * 3), ("color_hi", ctypes.c_float * 3),
                ("light_dir", ctypes.c_float * 3), ("light_rgb", ctypes.c_float * 3), ("env_rgb", ctypes.c_float * 3),
                ("max_bounces", ctypes.c_int32)]


def vpt_scene_struct(d: dict) -> "wrls_vpt_scene":
    """The C struct of a scene given as a dict of its fields (synth.vpt_scene)."""
    import numpy as np
    sc = wrls_vpt_scene()
    sc.struct_size = ctypes.sizeof(wrls_vpt_scene)
    sc.seed[0], sc.seed[1] = int(d["seed"]) & 0xFFFFFFFF, int(d["seed_hi"]) & 0xFFFFFFFF
    for name, n in (("eye", 3), ("color_lo", 3), ("color_hi", 3), ("light_dir", 3), ("light_rgb", 3),
                    ("env_rgb", 3), ("inv_view_proj", 16), ("blobs", 80)):
        getattr(sc, name)[:] = [float(v) for v in np.asarray(d[name], np.float32).reshape(n)]
    sc.n_blobs, sc.max_bounces = int(d["n_blobs"]), int(d["max_bounces"])
    sc.mu_max, sc.tf_lo, sc.tf_hi, sc.albedo = float(d["mu_max"]), float(d["tf_lo"]), float(d["tf_hi"]), float(d["albedo"])
    return sc


class wrls_frame_io(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("radiance", ctypes.c_void_p),
                ("variance", ctypes.c_void_p), ("features", ctypes.c_void_p),
                ("motion", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class wrls_state_stats(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_uint64), ("p_trace_max", ctypes.c_double),
                ("p_trace_mean", ctypes.c_double), ("p_diag_min", ctypes.c_double),
                ("nonfinite", ctypes.c_uint64)]


_lib = None


def lib():
    """Load libwrls.so (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libwrls.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i, P = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(wrls_params)
    sig = {
        "wrls_params_default": (None, [P]),
        "wrls_state_bytes": (ctypes.c_size_t, [i, i, P]),
        "wrls_stream_create": (i, [i, i, P, ctypes.POINTER(vp)]),
        "wrls_stream_set_cuda_stream": (i, [vp, vp]),
        "wrls_denoise_frame": (i, [vp, vp, vp, vp, vp, vp]),
        "wrls_denoise_frame_host": (i, [vp, vp, vp, vp, vp, vp]),
        "wrls_stream_reset": (i, [vp]),
        "wrls_stream_destroy": (None, [vp]),
        "wrls_stream_read_state": (i, [vp, vp]),
        "wrls_stream_write_state": (i, [vp, vp]),
        "wrls_stream_state_stats": (i, [vp, ctypes.POINTER(wrls_state_stats)]),
        "wrls_stream_frames": (ctypes.c_uint64, [vp]),
        "wrls_last_error": (ctypes.c_char_p, []),
        "wrls_stream_enable_timing": (i, [vp, i]),
        "wrls_stream_check": (i, [vp]),
        "wrls_stream_autotune": (i, [vp, vp, i, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]),
        "wrls_stream_set_blend_config": (i, [vp, i]),
        "wrls_stream_set_debug": (i, [vp, ctypes.c_uint32]),
        "wrls_stream_kernel_times": (i, [vp, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
        "wrls_batch_create": (i, [i, ctypes.POINTER(vp)]),
        "wrls_batch_set_cuda_stream": (i, [vp, vp]),
        "wrls_batch_tick": (i, [vp, ctypes.POINTER(wrls_frame_io), i]),
        "wrls_batch_destroy": (None, [vp]),
        "wrls_batch_tick_static": (i, [ctypes.POINTER(wrls_frame_io), i, vp]),
        "wrls_denoise_batch": (i, [ctypes.POINTER(vp), ctypes.POINTER(wrls_frame_io), i]),
        "wrls_denoise_sequence": (i, [vp, ctypes.POINTER(wrls_frame_io), i]),
        "wrls_denoise_sequence_host": (i, [vp, ctypes.POINTER(wrls_frame_io), i]),
        "wrls_stream_set_overlap": (i, [vp, i]),
        "wrls_recon_params_default": (None, [ctypes.POINTER(wrls_recon_params)]),
        "wrls_reconstruct": (i, [i, i, i, vp, ctypes.POINTER(wrls_recon_params), vp, vp, vp]),
        "wrls_velocity_from_world": (i, [i, i, vp, ctypes.POINTER(ctypes.c_float), i, vp, vp]),
        "wrls_render_vpt": (i, [ctypes.POINTER(wrls_vpt_scene), i, i, i, ctypes.c_uint32, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream_handle(cs) -> Optional[int]:
    if cs is None:
        return None
    if isinstance(cs, int):
        return cs
    return int(cs.cuda_stream)


def _check(status: int) -> None:
    if status != WRLS_OK:
        raise WrlsError(status, lib().wrls_last_error().decode(errors="replace"))


# --- C-named entry points ---------------------------------------------------------------

def wrls_params_default(**overrides) -> wrls_params:
    p = wrls_params()
    lib().wrls_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


def wrls_state_bytes(width: int, height: int, params: Optional[wrls_params] = None) -> int:
    p = params if params is not None else wrls_params_default()
    return int(lib().wrls_state_bytes(int(width), int(height), ctypes.byref(p)))


def wrls_stream_create(width: int, height: int, params: Optional[wrls_params] = None) -> int:
    p = params if params is not None else wrls_params_default()
    h = ctypes.c_void_p()
    _check(lib().wrls_stream_create(int(width), int(height), ctypes.byref(p), ctypes.byref(h)))
    return int(h.value)


def wrls_stream_set_cuda_stream(stream: int, cuda_stream) -> None:
    _check(lib().wrls_stream_set_cuda_stream(stream, _stream_handle(cuda_stream)))


def wrls_denoise_frame(stream: int, radiance, variance, features, motion, out) -> None:
    _check(lib().wrls_denoise_frame(stream, _ptr(radiance), _ptr(variance), _ptr(features),
                                    _ptr(motion), _ptr(out)))


def wrls_denoise_frame_host(stream: int, radiance, variance, features, motion, out) -> None:
    _check(lib().wrls_denoise_frame_host(stream, _ptr(radiance), _ptr(variance), _ptr(features),
                                         _ptr(motion), _ptr(out)))


def wrls_denoise_sequence(stream: int, frames: Sequence[tuple]) -> None:
    """frames: sequence of (radiance, variance, features, motion, out) of consecutive frames."""
    arr = (wrls_frame_io * max(1, len(frames)))()
    for k, (rad, var, feat, mot, out) in enumerate(frames):
        arr[k] = wrls_frame_io(stream, _ptr(rad), _ptr(var), _ptr(feat), _ptr(mot), _ptr(out))
    _check(lib().wrls_denoise_sequence(stream, arr, len(frames)))


def wrls_denoise_sequence_host(stream: int, frames: Sequence[tuple]) -> None:
    """frames: sequence of (radiance, variance, features, motion, out) HOST tensors (pinned)."""
    arr = (wrls_frame_io * max(1, len(frames)))()
    for k, (rad, var, feat, mot, out) in enumerate(frames):
        arr[k] = wrls_frame_io(stream, _ptr(rad), _ptr(var), _ptr(feat), _ptr(mot), _ptr(out))
    _check(lib().wrls_denoise_sequence_host(stream, arr, len(frames)))


def wrls_stream_set_overlap(stream: int, blend_ctas_per_sm: int) -> None:
    _check(lib().wrls_stream_set_overlap(stream, int(blend_ctas_per_sm)))


def wrls_recon_params_default(**overrides) -> wrls_recon_params:
    p = wrls_recon_params()
    lib().wrls_recon_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def wrls_reconstruct(samples, radiance, variance=None, params: Optional[wrls_recon_params] = None,
                     cuda_stream=None) -> None:
    """samples: device tensor (spp, 5, H, W) f32 (r, g, b, ox, oy); radiance (3, H, W) and
    optional variance (H, W) outputs."""
    spp, _, h, w = samples.shape
    p = params if params is not None else wrls_recon_params_default()
    _check(lib().wrls_reconstruct(int(w), int(h), int(spp), _ptr(samples), ctypes.byref(p), _ptr(radiance),
                                  _ptr(variance), _stream_handle(cuda_stream)))


def wrls_velocity_from_world(world, prev_view_proj, motion, miss_policy: int = 0, cuda_stream=None) -> None:
    """world: device tensor (3, H, W) f32; prev_view_proj: 4x4 row-major (host, any array
    type); motion (2, H, W) output."""
    _, h, w = world.shape
    m = (ctypes.c_float * 16)(*[float(v) for v in list(__import__("numpy").asarray(prev_view_proj).reshape(16))])
    _check(lib().wrls_velocity_from_world(int(w), int(h), _ptr(world), m, int(miss_policy), _ptr(motion),
                                          _stream_handle(cuda_stream)))


def wrls_render_vpt(scene, samples, world, features=None, frame: int = 0, cuda_stream=None) -> None:
    """scene: dict (synth.vpt_scene) or wrls_vpt_scene; samples (spp, 5, H, W), world (3, H, W),
    optional features (7, H, W) device tensors."""
    sc = scene if isinstance(scene, wrls_vpt_scene) else vpt_scene_struct(scene)
    spp, _, h, w = samples.shape
    _check(lib().wrls_render_vpt(ctypes.byref(sc), int(w), int(h), int(spp), int(frame) & 0xFFFFFFFF, _ptr(samples),
                                 _ptr(world), _ptr(features), _stream_handle(cuda_stream)))


def wrls_stream_reset(stream: int) -> None:
    _check(lib().wrls_stream_reset(stream))


def wrls_stream_destroy(stream: Optional[int]) -> None:
    if stream:
        lib().wrls_stream_destroy(stream)


def wrls_stream_read_state(stream: int, dst) -> None:
    _check(lib().wrls_stream_read_state(stream, _ptr(dst)))


def wrls_stream_write_state(stream: int, src) -> None:
    _check(lib().wrls_stream_write_state(stream, _ptr(src)))


def wrls_stream_state_stats(stream: int) -> dict:
    """State health: frames, trace(P) max / mean, smallest P diagonal, non-finite values."""
    st = wrls_state_stats()
    _check(lib().wrls_stream_state_stats(stream, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in wrls_state_stats._fields_}


def wrls_stream_frames(stream: int) -> int:
    return int(lib().wrls_stream_frames(stream))


BLEND_CONFIGS = 10


def wrls_stream_autotune(stream: int, out, reps: int = 5):
    """Time every blend tile configuration; returns (per-config ms list, chosen index)."""
    times = (ctypes.c_float * BLEND_CONFIGS)()
    chosen = ctypes.c_int()
    _check(lib().wrls_stream_autotune(stream, _ptr(out), int(reps), times, ctypes.byref(chosen)))
    return [float(t) for t in times], int(chosen.value)


WRLS_DEBUG_WITHHOLD_STAGE_COPY = 1
WRLS_DEBUG_NO_THIRD_COPY = 2


def wrls_stream_set_debug(stream: int, flags: int) -> None:
    """Test hooks: WRLS_DEBUG_WITHHOLD_STAGE_COPY makes the update kernel's bounded wait expire;
    WRLS_DEBUG_NO_THIRD_COPY (before the first sequence call) keeps the sequence entries on
    two state copies."""
    _check(lib().wrls_stream_set_debug(stream, int(flags)))


def wrls_stream_set_blend_config(stream: int, config: int) -> None:
    _check(lib().wrls_stream_set_blend_config(stream, int(config)))


def wrls_stream_check(stream: int) -> None:
    """Synchronise and raise WrlsError if a kernel's bounded wait gave up."""
    _check(lib().wrls_stream_check(stream))


def wrls_stream_enable_timing(stream: int, enable: bool = True) -> None:
    _check(lib().wrls_stream_enable_timing(stream, 1 if enable else 0))


def wrls_stream_kernel_times(stream: int):
    """(update_ms, blend_ms, frames) summed since the last call."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    _check(lib().wrls_stream_kernel_times(stream, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
    return float(a.value), float(b.value), int(n.value)


def wrls_last_error() -> str:
    return lib().wrls_last_error().decode(errors="replace")


def wrls_batch_create(max_streams: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().wrls_batch_create(int(max_streams), ctypes.byref(h)))
    return int(h.value)


def wrls_batch_set_cuda_stream(batch: int, cuda_stream) -> None:
    _check(lib().wrls_batch_set_cuda_stream(batch, _stream_handle(cuda_stream)))


def wrls_batch_tick(batch: int, frames: Sequence[tuple]) -> None:
    """frames: sequence of (stream, radiance, variance, features, motion, out)."""
    arr = (wrls_frame_io * len(frames))()
    for k, (s, rad, var, feat, mot, out) in enumerate(frames):
        arr[k] = wrls_frame_io(s, _ptr(rad), _ptr(var), _ptr(feat), _ptr(mot), _ptr(out))
    _check(lib().wrls_batch_tick(batch, arr, len(frames)))


STATIC_BATCH_MAX = 16


def wrls_batch_tick_static(frames: Sequence[tuple], cuda_stream=None) -> None:
    """The batched tick that allocates nothing (work table in a static device array).
    frames: sequence of (stream, radiance, variance, features, motion, out)."""
    arr = (wrls_frame_io * max(1, len(frames)))()
    for k, (s, rad, var, feat, mot, out) in enumerate(frames):
        arr[k] = wrls_frame_io(s, _ptr(rad), _ptr(var), _ptr(feat), _ptr(mot), _ptr(out))
    _check(lib().wrls_batch_tick_static(arr, len(frames), _stream_handle(cuda_stream)))


def wrls_denoise_batch(frames: Sequence[tuple]) -> None:
    """One batched tick on the library's executor. frames: (stream, radiance, variance,
    features, motion, out)."""
    n = len(frames)
    hs = (ctypes.c_void_p * max(1, n))()
    arr = (wrls_frame_io * max(1, n))()
    for k, (s, rad, var, feat, mot, out) in enumerate(frames):
        hs[k] = s
        arr[k] = wrls_frame_io(s, _ptr(rad), _ptr(var), _ptr(feat), _ptr(mot), _ptr(out))
    _check(lib().wrls_denoise_batch(hs, arr, n))


def wrls_batch_destroy(batch: Optional[int]) -> None:
    if batch:
        lib().wrls_batch_destroy(batch)


# --- convenience wrapper ---------------------------------------------------------------------

class Stream:
    """Owns one wrls_stream; frames are denoised on the given torch CUDA stream."""

    def __init__(self, width: int, height: int, params: Optional[wrls_params] = None, cuda_stream=None):
        self.width, self.height = int(width), int(height)
        self.params = params if params is not None else wrls_params_default()
        self.handle = wrls_stream_create(width, height, self.params)
        if cuda_stream is not None:
            wrls_stream_set_cuda_stream(self.handle, cuda_stream)

    def set_cuda_stream(self, cuda_stream) -> None:
        wrls_stream_set_cuda_stream(self.handle, cuda_stream)

    def denoise(self, radiance, motion, out, variance=None, features=None) -> None:
        wrls_denoise_frame(self.handle, radiance, variance, features, motion, out)

    def reset(self) -> None:
        wrls_stream_reset(self.handle)

    def read_state(self, dst) -> None:
        wrls_stream_read_state(self.handle, dst)

    def write_state(self, src) -> None:
        wrls_stream_write_state(self.handle, src)

    @property
    def state_planes(self) -> int:
        """Planes written by read_state: 25 on the paper's path, 3d + d(d+1)/2 + 3 with the
        extended predictor of dimension d."""
        p = self.params
        if p.n_gbuf > 0 or p.weight_mode == 2 or p.reproj_filter == 1:
            d = (4 if p.feature_mode == 0 else 1) + p.n_gbuf
            return 3 * d + d * (d + 1) // 2 + 3
        return 25

    def close(self) -> None:
        if self.handle:
            wrls_stream_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
