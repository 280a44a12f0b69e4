"""Parity of the extended CUDA path (G-buffer predictor entries up to d = 8, sample-variance
weight, nearest-pixel reprojection) with the extended FP64 oracle (oracle/wrls_oracle_ext.c),
through the C ABI, on the same seeded inputs: per-pixel relative error <= 1e-3 on the
denoised colour and on the temporal feature z, every pixel of every frame."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import REL_TOL, cpu_frames, ext_params_from, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    W.lib()


def params(**kw):
    kw.setdefault("n_features", synth.N_FEATURES)
    return W.wrls_params_default(**kw)


def run_ext(frames, width, height, p, hooks=None, tol=REL_TOL, host=False):
    s = W.Stream(width, height, p)
    st = O.OracleExtStream(width, height, ext_params_from(p))
    d = st.params.dim
    zoff = 3 * d + d * (d + 1) // 2
    assert s.state_planes == zoff + 3
    out = torch.empty(3, height, width, device="cuda")
    state = torch.empty(s.state_planes, height, width, device="cuda")
    h_out = torch.empty(3, height, width).pin_memory() if host else None
    errs = []
    for t, f in enumerate(frames):
        rad, mot = f["radiance"].clone(), f["motion"].clone()
        var, feat = f["variance"].clone(), f["features"].clone()
        if hooks is not None:
            rad, mot, var, feat = hooks(t, rad, mot, var, feat)
        if host:
            pinned = [x.pin_memory() for x in (rad, var, feat, mot)]  # alive until the sync
            W.wrls_denoise_frame_host(s.handle, *pinned, h_out)
            torch.cuda.synchronize()
            got = h_out.numpy().copy()
        else:
            s.denoise(rad.cuda(), mot.cuda(), out, variance=var.cuda(), features=feat.cuda())
            torch.cuda.synchronize()
            got = out.cpu().numpy()
        ref, _, _ = st.frame(rad.numpy(), mot.numpy(), var.numpy(), feat.numpy())
        s.read_state(state)
        e = rel_err(got, ref)
        ez = rel_err(state[zoff:zoff + 3].cpu().numpy(), st.z_planes())
        errs.append(max(e, ez))
        assert e <= tol and ez <= tol, "frame %d: out err %.3g, z err %.3g" % (t, e, ez)
    W.wrls_stream_check(s.handle)
    s.close()
    return errs


@pytest.mark.parametrize("n_gbuf", [1, 2, 3, 4])
def test_gbuffer_predictor_orbit_ragged(n_gbuf):
    spec = synth.SceneSpec(97, 61, 24, seed=41 + n_gbuf, motion="orbit", firefly_frac=0.05)
    errs = run_ext(cpu_frames(spec), spec.width, spec.height, params(n_gbuf=n_gbuf))
    print("n_gbuf", n_gbuf, "max err %.3g" % max(errs))


def test_gbuffer_predictor_d8_120_frames_with_edits():
    spec = synth.SceneSpec(130, 70, 120, seed=46, motion="pan", firefly_frac=0.05,
                           tf_edit_frame=60, light_move_frame=90)
    errs = run_ext(cpu_frames(spec), spec.width, spec.height, params(n_gbuf=4))
    print("d = 8, 120 frames: max err %.3g" % max(errs))


@pytest.mark.parametrize("mode", ["nf_g2", "var", "var_nf", "nearest", "nearest_g2", "blend_own_g3",
                                  "temporal_g2", "passthrough_g1", "guard_g4", "noclamp_var", "rls_nf_g4"])
def test_extended_modes(mode):
    kw = {"nf_g2": dict(feature_mode=1, n_gbuf=2), "var": dict(weight_mode=2),
          "var_nf": dict(weight_mode=2, feature_mode=1), "nearest": dict(reproj_filter=1),
          "nearest_g2": dict(reproj_filter=1, n_gbuf=2), "blend_own_g3": dict(blend_mode=1, n_gbuf=3),
          "temporal_g2": dict(radius=0, n_gbuf=2), "passthrough_g1": dict(init_mode=1, n_gbuf=1),
          "guard_g4": dict(p_trace_max=8.0, n_gbuf=4), "noclamp_var": dict(clamp_mode=1, weight_mode=2),
          "rls_nf_g4": dict(weight_mode=1, feature_mode=1, n_gbuf=4)}[mode]
    spec = synth.SceneSpec(83, 45, 16, seed=47, motion="orbit", firefly_frac=0.05)
    run_ext(cpu_frames(spec), spec.width, spec.height, params(**kw))


def test_missing_values_in_samples_variance_and_gbuffers():
    """Non-finite radiance (missing sample), non-finite or negative variance (weight 0 with
    the variance weight), non-finite G-buffer values (entry 0, weight 0), NaN motion
    (restart)."""
    spec = synth.SceneSpec(64, 40, 10, seed=48, motion="orbit")

    def hooks(t, rad, mot, var, feat):
        rad[1, 3, 5] = float("nan")
        rad[:, 20, 30] = float("inf")
        var[7, 7] = float("nan")
        var[8, 9] = -1.0
        feat[0, 10, 11] = float("nan")
        feat[2, 30, 40] = float("-inf")
        mot[0, 5, 50] = float("nan")
        return rad, mot, var, feat
    run_ext(cpu_frames(spec), spec.width, spec.height, params(weight_mode=2, n_gbuf=3), hooks=hooks)


def test_host_entry_copies_variance_and_features():
    spec = synth.SceneSpec(72, 40, 6, seed=49, motion="pan", firefly_frac=0.05)
    run_ext(cpu_frames(spec), spec.width, spec.height, params(weight_mode=2, n_gbuf=4), host=True)


def test_full_hd_d8_sampled_frames():
    """1920 x 1080 (the benchmark size), d = 8: every pixel of 4 frames."""
    spec = synth.SceneSpec(1920, 1080, 4, seed=50, motion="pan", firefly_frac=0.05)
    errs = run_ext(cpu_frames(spec), spec.width, spec.height, params(n_gbuf=4))
    print("1080p d = 8: max err %.3g" % max(errs))


def test_paper_path_equals_extended_path_for_d4():
    """Variance weight off, bilinear, no G-buffer entries: the extended kernels are not
    selected; with the variance weight selected but h huge (w ~ 1) the extended kernels and
    the fast kernels in RLS mode agree to the parity tolerance."""
    spec = synth.SceneSpec(80, 48, 12, seed=51, motion="orbit", firefly_frac=0.05)
    frames = cpu_frames(spec)
    a = W.Stream(spec.width, spec.height, params(weight_mode=1))
    b = W.Stream(spec.width, spec.height, params(weight_mode=2, h=1e6))
    oa = torch.empty(3, spec.height, spec.width, device="cuda")
    ob = torch.empty_like(oa)
    for f in frames:
        rad, mot = f["radiance"].cuda(), f["motion"].cuda()
        a.denoise(rad, mot, oa)
        b.denoise(rad, mot, ob, variance=f["variance"].cuda())
        torch.cuda.synchronize()
        assert rel_err(ob.cpu().numpy(), oa.cpu().numpy()) <= REL_TOL
    a.close()
    b.close()


def test_extended_streams_are_rejected_by_batched_ticks():
    s = W.Stream(64, 32, params(n_gbuf=2))
    b = W.wrls_batch_create(2)
    x = torch.zeros(3, 32, 64, device="cuda")
    m = torch.zeros(2, 32, 64, device="cuda")
    o = torch.empty_like(x)
    g = torch.zeros(7, 32, 64, device="cuda")
    with pytest.raises(W.WrlsError) as e:
        W.wrls_batch_tick(b, [(s.handle, x, None, g, m, o)])
    assert e.value.status == W.WRLS_ERR_INVALID_ARG
    with pytest.raises(W.WrlsError):
        W.wrls_batch_tick_static([(s.handle, x, None, g, m, o)])
    with pytest.raises(W.WrlsError):  # the G-buffer planes are required
        s.denoise(x, m, o)
    W.wrls_batch_destroy(b)
    s.close()
