"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/wrls.h
declares; host-only entry points behave (no GPU needed)."""
import os
import re

import pytest

from paper_2106_08034_gb300 import build as B
from paper_2106_08034_gb300 import wrls as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "wrls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    names = set(re.findall(r"\b(wrls_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return W.lib()


def test_header_and_binding_agree():
    assert _declared_functions() == sorted(W.EXPORTED)


def test_header_constants_match_the_binding():
    src = open(os.path.join(ROOT, "include", "wrls.h")).read()
    m = re.search(r"#define\s+WRLS_STATIC_BATCH_MAX\s+(\d+)", src)
    assert m and int(m.group(1)) == W.STATIC_BATCH_MAX
    for name in ("WRLS_DEBUG_WITHHOLD_STAGE_COPY", "WRLS_DEBUG_NO_THIRD_COPY"):
        m = re.search(r"#define\s+%s\s+(\d+)u" % name, src)
        assert m and int(m.group(1)) == getattr(W, name), name


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_params_default_are_the_papers(lib):
    p = W.wrls_params_default()
    assert p.struct_size == __import__("ctypes").sizeof(W.wrls_params)
    assert abs(p.lambda_ - 0.998) < 1e-7 and p.h == 0.75 and p.alpha == 0.75 and p.radius == 2


def test_state_bytes(lib):
    p = W.wrls_params_default()
    b32 = W.wrls_state_bytes(1920, 1080, p)
    assert b32 >= 2 * 25 * 4 * 1920 * 1080 and b32 < 2 * 25 * 4 * 1920 * 1088 + 4096
    p.state_precision = W.WRLS_STATE_BF16
    b16 = W.wrls_state_bytes(1920, 1080, p)
    assert b16 >= 2 * 52 * 1920 * 1080 and b16 < 0.6 * b32
    assert W.wrls_state_bytes(0, 10, p) == 0 and W.wrls_state_bytes(10, 20000, p) == 0


def test_invalid_arguments_are_rejected_on_the_host(lib):
    with pytest.raises(W.WrlsError) as e:
        W.wrls_stream_create(0, 10)
    assert e.value.status == W.WRLS_ERR_INVALID_ARG and "width" in W.wrls_last_error()
    p = W.wrls_params_default()
    p.radius = 3
    with pytest.raises(W.WrlsError):
        W.wrls_stream_create(8, 8, p)
    p = W.wrls_params_default()
    p.struct_size = 4
    with pytest.raises(W.WrlsError):
        W.wrls_stream_create(8, 8, p)
    with pytest.raises(W.WrlsError):
        W.wrls_batch_create(0)
    assert lib.wrls_denoise_frame(None, None, None, None, None, None) == W.WRLS_ERR_INVALID_ARG
    W.wrls_stream_destroy(0)
    W.wrls_batch_destroy(0)


def test_extended_path_parameters_are_checked_on_the_host(lib):
    """G-buffer predictor entries need n_features >= n_gbuf and at most 4 entries; the
    extended path needs the binary32 state; weight_mode and reproj_filter are range-checked."""
    bad = [dict(n_gbuf=2, n_features=1), dict(n_gbuf=5, n_features=7), dict(n_gbuf=-1),
           dict(weight_mode=3), dict(reproj_filter=2),
           dict(n_gbuf=1, n_features=1, state_precision=W.WRLS_STATE_BF16),
           dict(weight_mode=2, state_precision=W.WRLS_STATE_F16),
           dict(reproj_filter=1, state_precision=W.WRLS_STATE_BF16)]
    for kw in bad:
        with pytest.raises(W.WrlsError) as e:
            W.wrls_stream_create(8, 8, W.wrls_params_default(**kw))
        assert e.value.status == W.WRLS_ERR_INVALID_ARG, kw


def test_extended_state_bytes(lib):
    """3d + d(d+1)/2 + 3 binary32 planes per pixel and copy: d = 8 -> 63 planes (252 B/px)."""
    base = W.wrls_state_bytes(640, 360, W.wrls_params_default())
    for kw, planes in [(dict(n_gbuf=4, n_features=7), 63), (dict(n_gbuf=1, n_features=1), 33),
                       (dict(weight_mode=2), 25), (dict(reproj_filter=1), 25),
                       (dict(n_gbuf=2, n_features=2, feature_mode=1), 18)]:
        b = W.wrls_state_bytes(640, 360, W.wrls_params_default(**kw))
        assert abs(b / base - planes / 25) < 1e-3, (kw, b, base)


def test_input_step_arguments_are_checked_on_the_host(lib):
    import ctypes
    p = W.wrls_recon_params_default()
    assert abs(p.sigma - 0.5) < 1e-7 and abs(p.radius - 1.5) < 1e-7
    bad = W.wrls_recon_params_default(radius=1.6)
    assert lib.wrls_reconstruct(8, 8, 1, 256, ctypes.byref(bad), 4096, None, None) == W.WRLS_ERR_INVALID_ARG
    assert lib.wrls_reconstruct(8, 8, 0, 256, ctypes.byref(p), 4096, None, None) == W.WRLS_ERR_INVALID_ARG
    p.struct_size = 3
    assert lib.wrls_reconstruct(8, 8, 1, 256, ctypes.byref(p), 4096, None, None) == W.WRLS_ERR_INVALID_ARG
    m = (ctypes.c_float * 16)(*([1.0] * 16))
    assert lib.wrls_velocity_from_world(8, 8, 256, m, 2, 4096, None) == W.WRLS_ERR_INVALID_ARG
    m[3] = float("inf")
    assert lib.wrls_velocity_from_world(8, 8, 256, m, 0, 4096, None) == W.WRLS_ERR_INVALID_ARG


def test_write_state_arguments_are_checked_on_the_host(lib):
    assert lib.wrls_stream_write_state(None, None) == W.WRLS_ERR_INVALID_ARG
    assert lib.wrls_stream_state_stats(None, None) == W.WRLS_ERR_INVALID_ARG


def test_denoise_batch_arguments_are_checked_on_the_host(lib):
    assert lib.wrls_denoise_batch(None, None, 1) == W.WRLS_ERR_INVALID_ARG
    import ctypes
    hs = (ctypes.c_void_p * 1)(None)
    arr = (W.wrls_frame_io * 1)()
    assert lib.wrls_denoise_batch(hs, arr, 0) == W.WRLS_ERR_INVALID_ARG
    assert lib.wrls_denoise_batch(hs, arr, 1) == W.WRLS_ERR_INVALID_ARG   # NULL stream
