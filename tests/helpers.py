"""Shared helpers of the tests: seeded inputs (CPU-generated, copied to the GPU), oracle
runs and the parity metric."""
import numpy as np
import torch

import oracle as O
from paper_2106_08034_gb300 import synth

# Parity gate of the FP32 path: per pixel, the relative error of its colour vector,
#   max_c |gpu_c - oracle_c| / max(max_c |oracle_c|, FLOOR),
# maximised over pixels and frames, must be <= REL_TOL. Colours are compared as vectors,
# as the paper does (Eq. 13 norms; Table 2 errors "considering color channels"): one
# channel of a large colour may cancel to near zero, and its error is judged at the scale
# of the pixel. FLOOR keeps near-black pixels from dominating the relative measure.
REL_TOL = 1e-3
FLOOR = 1e-2


def rel_err(gpu, ref):
    """Max per-pixel relative error of (C, H, W) colour arrays (vectors along axis 0)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    num = np.max(np.abs(gpu - ref), axis=0)
    den = np.maximum(np.max(np.abs(ref), axis=0), FLOOR)
    return float(np.max(num / den))


def relmse(x, truth):
    x = np.asarray(x, np.float64)
    t = np.asarray(truth, np.float64)
    return float(np.mean((x - t) ** 2 / (t * t + 1e-2)))


def oracle_params_from(p):
    """OracleParams with the same settings as a wrls_params struct."""
    return O.OracleParams(lambda_=float(np.float32(p.lambda_)), h=float(np.float32(p.h)),
                          alpha=float(np.float32(p.alpha)), eps=float(np.float32(p.eps)),
                          p0_delta=float(np.float32(p.p0_delta)), sigma_s=float(np.float32(p.sigma_s)),
                          h_s=float(np.float32(p.h_s)), p_trace_max=float(np.float32(p.p_trace_max)),
                          radius=p.radius, weight_mode=p.weight_mode, clamp_mode=p.clamp_mode,
                          blend_mode=p.blend_mode, feature_mode=p.feature_mode, init_mode=p.init_mode)


def ext_params_from(p):
    """OracleExtParams with the same settings as a wrls_params struct (extended path)."""
    base = oracle_params_from(p)
    return O.OracleExtParams(**{**base.__dict__, "n_gbuf": p.n_gbuf, "reproj_filter": p.reproj_filter})


def cpu_frames(spec, count=None):
    sc = synth.Scene(spec)
    T = spec.frames if count is None else count
    return [sc.frame(t) for t in range(T)]


def oracle_z_planes(st):
    return st.z.reshape(st.H, st.W, 3).transpose(2, 0, 1)


def rel_err_channel(gpu, ref):
    """Max per-channel relative error |gpu_c - ref_c| / max(|ref_c|, FLOOR) of (C, H, W) colour
    arrays: the stricter channel-by-channel form, reported beside the per-pixel parity metric."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), FLOOR)))
