"""wRLS denoiser ORACLE: plain FP64 CPU implementation in ``wrls_oracle.c``.

Test infrastructure only. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA library and never imports it.

``build()`` compiles ``wrls_oracle.c`` (the paper's predictor p = [1, z], d = 4) and
``wrls_oracle_ext.c`` (any d <= 8: G-buffer predictor entries, sample-variance weight,
nearest-pixel reprojection), ``wrls_oracle_upstream.c`` (pixel reconstruction filter,
velocity from first-collision world positions) and ``wrls_oracle_vpt.c`` (delta-tracking
volumetric path tracer) with gcc (``-O2 -ffp-contract=off -fopenmp``) into
``oracle/_build/libwrls_oracle.so``; ``OracleStream`` and ``OracleExtStream`` run frames
through them.
The constants in ``OracleParams`` defaults are the paper's where it gives one
(lambda = 0.998 in Sec. 5.2, h = 0.75 in Sec. 5.3, alpha = 0.75 in Sec. 6, a 5x5 blend
window in Sec. 5.3) and the readings of the C file's header elsewhere.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wrls_oracle.c")
_SRC_EXT = os.path.join(_HERE, "wrls_oracle_ext.c")
_SRC_UP = os.path.join(_HERE, "wrls_oracle_upstream.c")
_SRC_VPT = os.path.join(_HERE, "wrls_oracle_vpt.c")
SOURCES = (_SRC, _SRC_EXT, _SRC_UP, _SRC_VPT)
_LIB = os.path.join(_HERE, "_build", "libwrls_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, gcc) if missing or older than its source."""
    newest = max(os.path.getmtime(p) for p in SOURCES)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, *SOURCES, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("h", ctypes.c_double), ("alpha", ctypes.c_double),
                ("eps", ctypes.c_double), ("p0_delta", ctypes.c_double),
                ("sigma_s", ctypes.c_double), ("h_s", ctypes.c_double),
                ("p_trace_max", ctypes.c_double),
                ("radius", ctypes.c_int), ("weight_mode", ctypes.c_int),
                ("clamp_mode", ctypes.c_int), ("blend_mode", ctypes.c_int),
                ("feature_mode", ctypes.c_int), ("init_mode", ctypes.c_int)]


@dataclasses.dataclass
class OracleParams:
    lambda_: float = 0.998     # Sec. 5.2 (Eq. 10)
    h: float = 0.75            # Sec. 5.3 (Eq. 13)
    alpha: float = 0.75        # Sec. 6 (Eq. 12)
    eps: float = 1e-4
    p0_delta: float = 1.0
    sigma_s: float = 1.0
    h_s: float = 0.75
    p_trace_max: float = 0.0
    radius: int = 2            # 5x5 window, Sec. 5.3
    weight_mode: int = 0       # 0 wRLS, 1 RLS
    clamp_mode: int = 0        # 0 3x3 clamp, 1 off
    blend_mode: int = 0        # 0 p_i beta_k, 1 p_k beta_k
    feature_mode: int = 0      # 0 p=[1,z], 1 p=[1]
    init_mode: int = 0         # 0 beta = 0, 1 feature pass-through

    def c(self) -> _Params:
        return _Params(*dataclasses.astuple(self))


class _ExtParams(ctypes.Structure):
    _fields_ = _Params._fields_ + [("n_gbuf", ctypes.c_int), ("reproj_filter", ctypes.c_int)]


@dataclasses.dataclass
class OracleExtParams(OracleParams):
    """Parameters of ``wrls_oracle_ext.c``: the paper's plus the alternatives it sets aside."""
    n_gbuf: int = 0            # G-buffer planes appended to the predictor (0..4)
    reproj_filter: int = 0     # 0 bilinear, 1 nearest pixel
    # weight_mode 2: sample-variance weight

    def c(self) -> _ExtParams:
        return _ExtParams(*dataclasses.astuple(self))

    @property
    def dim(self) -> int:
        return (4 if self.feature_mode == 0 else 1) + self.n_gbuf


class _VptScene(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32 * 2), ("eye", ctypes.c_float * 3), ("inv_view_proj", ctypes.c_float * 16),
                ("n_blobs", ctypes.c_int), ("blobs", ctypes.c_float * 80), ("mu_max", ctypes.c_float),
                ("tf_lo", ctypes.c_float), ("tf_hi", ctypes.c_float), ("albedo", ctypes.c_float),
                ("color_lo", ctypes.c_float * 3), ("color_hi", ctypes.c_float * 3),
                ("light_dir", ctypes.c_float * 3), ("light_rgb", ctypes.c_float * 3),
                ("env_rgb", ctypes.c_float * 3), ("max_bounces", ctypes.c_int)]


def _vpt_scene(d: dict) -> _VptScene:
    sc = _VptScene()
    sc.seed[0], sc.seed[1] = int(d["seed"]) & 0xFFFFFFFF, int(d["seed_hi"]) & 0xFFFFFFFF
    for name, n in (("eye", 3), ("color_lo", 3), ("color_hi", 3), ("light_dir", 3), ("light_rgb", 3),
                    ("env_rgb", 3)):
        arr = np.asarray(d[name], np.float32).reshape(n)
        getattr(sc, name)[:] = [float(v) for v in arr]
    sc.inv_view_proj[:] = [float(v) for v in np.asarray(d["inv_view_proj"], np.float32).reshape(16)]
    sc.blobs[:] = [float(v) for v in np.asarray(d["blobs"], np.float32).reshape(80)]
    sc.n_blobs, sc.max_bounces = int(d["n_blobs"]), int(d["max_bounces"])
    sc.mu_max, sc.tf_lo, sc.tf_hi, sc.albedo = float(d["mu_max"]), float(d["tf_lo"]), float(d["tf_hi"]), float(d["albedo"])
    return sc


def lib():
    """Load the oracle library (``WRLS_ORACLE_LIB`` selects another build of the same
    source, which the mutation tests use to load deliberately broken copies)."""
    global _lib
    if _lib is None:
        override = os.environ.get("WRLS_ORACLE_LIB")
        _lib = ctypes.CDLL(override if override else build())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        _lib.wrls_oracle_frame.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, dp, dp, dp, fp, fp, dp, dp, dp, dp, dp,
                                           ctypes.POINTER(ctypes.c_ubyte)]
        _lib.wrls_oracle_frame.restype = ctypes.c_int
        _lib.wrls_oracle_blend.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                           dp, dp, dp]
        _lib.wrls_oracle_blend.restype = ctypes.c_int
        _lib.wrls_oracle_ext_frame.argtypes = [ctypes.POINTER(_ExtParams), ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, dp, dp, dp, fp, fp, fp, fp, dp, dp, dp, dp,
                                               dp, ctypes.POINTER(ctypes.c_ubyte)]
        _lib.wrls_oracle_ext_frame.restype = ctypes.c_int
        _lib.wrls_oracle_ext_blend.argtypes = [ctypes.POINTER(_ExtParams), ctypes.c_int, ctypes.c_int,
                                               dp, dp, fp, dp]
        _lib.wrls_oracle_ext_blend.restype = ctypes.c_int
        _lib.wrls_oracle_ext_dim.argtypes = [ctypes.POINTER(_ExtParams)]
        _lib.wrls_oracle_ext_dim.restype = ctypes.c_int
        _lib.wrls_oracle_reconstruct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, ctypes.c_double,
                                                 ctypes.c_double, dp, dp]
        _lib.wrls_oracle_reconstruct.restype = ctypes.c_int
        _lib.wrls_oracle_velocity.argtypes = [ctypes.c_int, ctypes.c_int, fp, dp, ctypes.c_int, dp]
        _lib.wrls_oracle_velocity.restype = ctypes.c_int
        _lib.wrls_oracle_render_vpt.argtypes = [ctypes.POINTER(_VptScene), ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_uint32, fp, fp, fp]
        _lib.wrls_oracle_render_vpt.restype = ctypes.c_int
        u32p = ctypes.POINTER(ctypes.c_uint32)
        _lib.wrls_oracle_philox.argtypes = [u32p, u32p, u32p]
        _lib.wrls_oracle_philox.restype = None
        _lib.wrls_oracle_set_threads.argtypes = [ctypes.c_int]
        _lib.wrls_oracle_get_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> None:
    lib().wrls_oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().wrls_oracle_get_threads())


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class OracleStream:
    """Per-stream oracle state (beta [n,3,4], full P [n,4,4], z [n,3]) across frames."""

    def __init__(self, width: int, height: int, params: Optional[OracleParams] = None):
        self.W, self.H = int(width), int(height)
        self.params = params or OracleParams()
        n = self.W * self.H
        self.beta = np.zeros((n, 3, 4))
        self.P = np.zeros((n, 4, 4))
        self.z = np.zeros((n, 3))
        self.need_reset = True

    def reset(self) -> None:
        self.need_reset = True

    def frame(self, radiance: np.ndarray, motion: np.ndarray):
        """Run one frame. radiance (3,H,W) f32, motion (2,H,W) f32.
        Returns (out (3,H,W) f64, w (H,W) f64, valid (H,W) bool)."""
        W, H = self.W, self.H
        rad = np.ascontiguousarray(radiance, dtype=np.float32)
        mot = np.ascontiguousarray(motion, dtype=np.float32)
        assert rad.shape == (3, H, W) and mot.shape == (2, H, W)
        n = W * H
        bn, Pn, zn = np.empty((n, 3, 4)), np.empty((n, 4, 4)), np.empty((n, 3))
        out = np.empty((3, H, W))
        w = np.empty((H, W))
        valid = np.empty((H, W), dtype=np.uint8)
        prm = self.params.c()
        rc = lib().wrls_oracle_frame(ctypes.byref(prm), W, H, int(self.need_reset),
                                     _dptr(self.beta), _dptr(self.P), _dptr(self.z),
                                     _fptr(rad), _fptr(mot), _dptr(bn), _dptr(Pn), _dptr(zn),
                                     _dptr(out), _dptr(w),
                                     valid.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        if rc != 0:
            raise ValueError("wrls_oracle_frame rejected its arguments")
        self.beta, self.P, self.z = bn, Pn, zn
        self.need_reset = False
        return out, w, valid.astype(bool)

    def z_planes(self) -> np.ndarray:
        return self.z.reshape(self.H, self.W, 3).transpose(2, 0, 1)


def blend(params: OracleParams, beta: np.ndarray, z: np.ndarray, width: int, height: int) -> np.ndarray:
    """The blend step alone on an explicit state: beta [n,3,4], z [n,3] -> out (3,H,W)."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = np.empty((3, height, width))
    prm = params.c()
    rc = lib().wrls_oracle_blend(ctypes.byref(prm), int(width), int(height), _dptr(beta), _dptr(z),
                                 _dptr(out))
    if rc != 0:
        raise ValueError("wrls_oracle_blend rejected its arguments")
    return out


def _fptr_opt(a: Optional[np.ndarray]):
    return None if a is None else _fptr(a)


class OracleExtStream:
    """Per-stream state of the extended oracle: beta [n,3,d], full P [n,d,d], z [n,3]."""

    def __init__(self, width: int, height: int, params: Optional[OracleExtParams] = None):
        self.W, self.H = int(width), int(height)
        self.params = params or OracleExtParams()
        d, n = self.params.dim, self.W * self.H
        self.beta = np.zeros((n, 3, d))
        self.P = np.zeros((n, d, d))
        self.z = np.zeros((n, 3))
        self.need_reset = True

    def reset(self) -> None:
        self.need_reset = True

    def frame(self, radiance: np.ndarray, motion: np.ndarray, variance: Optional[np.ndarray] = None,
              gbuf: Optional[np.ndarray] = None):
        """One frame. radiance (3,H,W), motion (2,H,W), variance (H,W) or None, gbuf
        (>= n_gbuf,H,W) or None, all f32. Returns (out (3,H,W) f64, w (H,W), valid (H,W))."""
        W, H, prm = self.W, self.H, self.params
        d, n = prm.dim, W * H
        rad = np.ascontiguousarray(radiance, dtype=np.float32)
        mot = np.ascontiguousarray(motion, dtype=np.float32)
        var = None if variance is None else np.ascontiguousarray(variance, dtype=np.float32).reshape(H, W)
        g = None
        if gbuf is not None and prm.n_gbuf > 0:
            g = np.ascontiguousarray(np.asarray(gbuf, dtype=np.float32)[:prm.n_gbuf])
            assert g.shape == (prm.n_gbuf, H, W)
        bn, Pn, zn = np.empty((n, 3, d)), np.empty((n, d, d)), np.empty((n, 3))
        out = np.empty((3, H, W))
        w = np.empty((H, W))
        valid = np.empty((H, W), dtype=np.uint8)
        c = prm.c()
        rc = lib().wrls_oracle_ext_frame(ctypes.byref(c), W, H, int(self.need_reset),
                                         _dptr(self.beta), _dptr(self.P), _dptr(self.z),
                                         _fptr(rad), _fptr(mot), _fptr_opt(var), _fptr_opt(g),
                                         _dptr(bn), _dptr(Pn), _dptr(zn), _dptr(out), _dptr(w),
                                         valid.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        if rc != 0:
            raise ValueError("wrls_oracle_ext_frame rejected its arguments")
        self.beta, self.P, self.z = bn, Pn, zn
        self.need_reset = False
        return out, w, valid.astype(bool)

    def z_planes(self) -> np.ndarray:
        return self.z.reshape(self.H, self.W, 3).transpose(2, 0, 1)


def reconstruct(samples: np.ndarray, sigma: float = 0.5, radius: float = 1.5, with_variance: bool = True):
    """Pixel reconstruction filter. samples (spp, 5, H, W) f32 (r, g, b, ox, oy).
    Returns (radiance (3,H,W) f64, variance (H,W) f64 or None)."""
    smp = np.ascontiguousarray(samples, dtype=np.float32)
    spp, five, H, W = smp.shape
    assert five == 5
    out = np.empty((3, H, W))
    var = np.empty((H, W)) if with_variance else None
    rc = lib().wrls_oracle_reconstruct(W, H, spp, _fptr(smp), float(sigma), float(radius), _dptr(out), _dptr(var))
    if rc != 0:
        raise ValueError("wrls_oracle_reconstruct rejected its arguments")
    return out, var


def velocity(world: np.ndarray, prev_view_proj: np.ndarray, miss_policy: int = 0) -> np.ndarray:
    """Backward motion (2,H,W) f64 from first-collision world positions (3,H,W) f32 and the
    previous frame's 4x4 view-projection matrix (row-major)."""
    wd = np.ascontiguousarray(world, dtype=np.float32)
    _, H, W = wd.shape
    M = np.ascontiguousarray(prev_view_proj, dtype=np.float64).reshape(16)
    mot = np.empty((2, H, W))
    rc = lib().wrls_oracle_velocity(W, H, _fptr(wd), _dptr(M), int(miss_policy), _dptr(mot))
    if rc != 0:
        raise ValueError("wrls_oracle_velocity rejected its arguments")
    return mot


def render_vpt(scene: dict, width: int, height: int, spp: int, frame: int = 0, features: bool = True):
    """Delta-tracking path tracer. Returns (samples (spp,5,H,W), world (3,H,W), features (7,H,W)
    or None), all f32."""
    sc = _vpt_scene(scene)
    smp = np.empty((spp, 5, height, width), np.float32)
    world = np.empty((3, height, width), np.float32)
    feat = np.empty((7, height, width), np.float32) if features else None
    rc = lib().wrls_oracle_render_vpt(ctypes.byref(sc), int(width), int(height), int(spp), int(frame) & 0xFFFFFFFF,
                                      _fptr(smp), _fptr(world), None if feat is None else _fptr(feat))
    if rc != 0:
        raise ValueError("wrls_oracle_render_vpt rejected its arguments")
    return smp, world, feat


def philox(counter, key):
    """Philox4x32-10 block of the oracle: 4 uint32 counter words, 2 key words -> 4 words."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().wrls_oracle_philox(c, k, o)
    return [int(v) for v in o]
