"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs. FP32 state: per-pixel relative error <= 1e-3 on the denoised colour and on the
temporal feature z, every pixel of every frame (helpers.rel_err: colour vectors, floor
1e-2)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import FLOOR, REL_TOL, cpu_frames, ext_params_from, oracle_params_from, oracle_z_planes, rel_err, relmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    W.lib()


def run_pair(frames, width, height, params=None, hooks=None, check_z=True, tol=REL_TOL, blend_config=None):
    """Denoise the frames with the GPU and with the oracle; assert parity every frame.
    Returns the per-frame max relative errors."""
    p = params if params is not None else W.wrls_params_default()
    s = W.Stream(width, height, p)
    if blend_config is not None:
        W.wrls_stream_set_blend_config(s.handle, blend_config)
    st = O.OracleStream(width, height, oracle_params_from(p))
    out = torch.empty(3, height, width, device="cuda")
    zbuf = torch.empty(W.N_STATE, height, width, device="cuda")
    errs = []
    for t, f in enumerate(frames):
        rad, mot = f["radiance"].clone(), f["motion"].clone()
        if hooks is not None:
            rad, mot = hooks(t, rad, mot)
        s.denoise(rad.cuda(), mot.cuda(), out)
        ref, _, _ = st.frame(rad.numpy(), mot.numpy())
        torch.cuda.synchronize()
        e = rel_err(out.cpu().numpy(), ref)
        ez = 0.0
        if check_z:
            s.read_state(zbuf)
            ez = rel_err(zbuf[22:25].cpu().numpy(), oracle_z_planes(st))
        errs.append(max(e, ez))
        assert e <= tol and ez <= tol, "frame %d: out err %.3g, z err %.3g" % (t, e, ez)
    W.wrls_stream_check(s.handle)
    s.close()
    return errs


def test_static_128x128_8f():
    spec = synth.static_128x128_8f()
    run_pair(cpu_frames(spec), spec.width, spec.height)


def test_pan_fireflies_ragged_tiles():
    spec = synth.SceneSpec(250, 150, 24, seed=31, motion="pan", firefly_frac=0.05)
    run_pair(cpu_frames(spec), spec.width, spec.height)


def test_orbit_edit_light_move_120_frames():
    spec = synth.SceneSpec(203, 117, 120, seed=32, motion="orbit", firefly_frac=0.05,
                           tf_edit_frame=60, light_move_frame=90)
    run_pair(cpu_frames(spec), spec.width, spec.height)


@pytest.mark.parametrize("mode", ["rls", "noclamp", "blend_own", "temporal_only", "radius1",
                                  "no_feature", "passthrough", "trace_guard", "lambda1"])
def test_modes(mode):
    kw = {"rls": dict(weight_mode=1), "noclamp": dict(clamp_mode=1), "blend_own": dict(blend_mode=1),
          "temporal_only": dict(radius=0), "radius1": dict(radius=1), "no_feature": dict(feature_mode=1),
          "passthrough": dict(init_mode=1), "trace_guard": dict(p_trace_max=3.9),
          "lambda1": {"lambda": 1.0}}[mode]
    p = W.wrls_params_default(**kw)
    spec = synth.SceneSpec(70, 45, 16, seed=33, motion="orbit", firefly_frac=0.05)
    run_pair(cpu_frames(spec), spec.width, spec.height, p)


@pytest.mark.parametrize("wh", [(1, 1), (1, 37), (41, 1), (2, 2), (33, 9), (32, 8), (64, 16)])
def test_degenerate_sizes(wh):
    w, h = wh
    spec = synth.SceneSpec(w, h, 6, seed=34, motion="orbit", firefly_frac=0.1)
    run_pair(cpu_frames(spec), w, h)


@pytest.mark.parametrize("wh", [(16384, 24), (24, 16384)])
def test_maximum_dimensions(wh):
    """The largest width and height the stream accepts (16384), every pixel of 3 frames
    against the oracle."""
    w, h = wh
    spec = synth.SceneSpec(w, h, 3, seed=37, motion="orbit", firefly_frac=0.05)
    run_pair(cpu_frames(spec), w, h, check_z=False)


def test_large_frame_sampled_crops():
    """8192 x 8192 (67 Mpx, 13.4 GB of binary32 state in two copies), static camera, 3 frames:
    sampled crops (corners, edges, centre) equal the oracle run on the crop plus a 3-pixel
    margin; with zero motion a pixel's output depends only on its 7 x 7 neighbourhood (3 x 3
    clamp box of each of the 5 x 5 blended models)."""
    w = h = 8192
    spec = synth.SceneSpec(w, h, 3, seed=38, motion="static", firefly_frac=0.05)
    sc = synth.Scene(spec)
    s = W.Stream(w, h)
    out = torch.empty(3, h, w, device="cuda")
    c, m = 40, 3
    corners = [(0, 0), (w - c, 0), (0, h - c), (w - c, h - c), (w // 2 - 17, h // 2 + 5), (w // 3, 0), (0, h // 3)]
    crops = []
    for (x0, y0) in corners:
        ax0, ay0 = max(x0 - m, 0), max(y0 - m, 0)
        ax1, ay1 = min(x0 + c + m, w), min(y0 + c + m, h)
        crops.append((x0, y0, ax0, ay0, ax1, ay1, O.OracleStream(ax1 - ax0, ay1 - ay0)))
    for t in range(spec.frames):
        f = sc.frame(t, device="cuda")
        s.denoise(f["radiance"], f["motion"], out)
        rad = f["radiance"]
        for (x0, y0, ax0, ay0, ax1, ay1, st) in crops:
            r = rad[:, ay0:ay1, ax0:ax1].cpu().numpy()
            ref, _, _ = st.frame(r, np.zeros((2,) + r.shape[1:], np.float32))
            got = out[:, y0:y0 + c, x0:x0 + c].cpu().numpy()
            exp = ref[:, y0 - ay0:y0 - ay0 + c, x0 - ax0:x0 - ax0 + c]
            assert rel_err(got, exp) <= REL_TOL, (t, x0, y0)
        del f, rad
    W.wrls_stream_check(s.handle)
    s.close()


@pytest.mark.parametrize("wh", [(72, 20), (75, 21), (130, 27), (200, 20)])
def test_two_wide_blend_at_its_smallest_sizes(wh):
    """Blend configurations 8 and 9 where their TMA boxes (72 or 80 columns x 12 or 20 rows)
    cover most or all of the image: binary32 against the oracle every frame; BF16 and FP16
    bitwise equal to the one-CTA-per-tile blend."""
    w, h = wh
    spec = synth.SceneSpec(w, h, 6, seed=35, motion="orbit", firefly_frac=0.05)
    fr = cpu_frames(spec)
    for cfg in (8, 9):
        s = W.Stream(w, h)
        W.wrls_stream_set_blend_config(s.handle, cfg)
        st = O.OracleStream(w, h, oracle_params_from(W.wrls_params_default()))
        out = torch.empty(3, h, w, device="cuda")
        for f in fr:
            s.denoise(f["radiance"].cuda(), f["motion"].cuda(), out)
            ref, _, _ = st.frame(f["radiance"].numpy(), f["motion"].numpy())
            assert rel_err(out.cpu().numpy(), ref) <= REL_TOL, cfg
        W.wrls_stream_check(s.handle)
        s.close()
    for prec in (1, 2):
        outs = []
        for cfg in (0, 8, 9):
            s = W.Stream(w, h, W.wrls_params_default(state_precision=prec))
            W.wrls_stream_set_blend_config(s.handle, cfg)
            out = torch.empty(3, h, w, device="cuda")
            for f in fr:
                s.denoise(f["radiance"].cuda(), f["motion"].cuda(), out)
            W.wrls_stream_check(s.handle)
            outs.append(out.cpu())
            s.close()
        assert torch.equal(outs[1], outs[0]) and torch.equal(outs[2], outs[0]), prec


@pytest.mark.parametrize("wh", [(1, 1), (1, 37), (41, 1), (33, 9)])
def test_degenerate_sizes_sequence_and_extended(wh):
    """The sequence entry (three state copies, blend on a second CUDA stream) and the extended
    path on degenerate images: sequence bitwise equal to per-frame calls, both at parity with
    the oracle."""
    w, h = wh
    spec = synth.SceneSpec(w, h, 6, seed=36, motion="orbit", firefly_frac=0.1)
    fr = cpu_frames(spec)
    p = W.wrls_params_default()
    ref = run_pair(fr, w, h, p)
    assert max(ref) <= REL_TOL
    per = []
    s = W.Stream(w, h, p)
    for f in fr:
        o = torch.empty(3, h, w, device="cuda")
        s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
        per.append(o)
    W.wrls_stream_check(s.handle)
    s.close()
    s = W.Stream(w, h, p)
    seq = [torch.empty(3, h, w, device="cuda") for _ in fr]
    W.wrls_denoise_sequence(s.handle, [(f["radiance"].cuda(), None, None, f["motion"].cuda(), seq[t])
                                       for t, f in enumerate(fr)])
    W.wrls_stream_check(s.handle)
    s.close()
    for a, b in zip(per, seq):
        assert torch.equal(a, b)
    pe = W.wrls_params_default(n_features=synth.N_FEATURES, n_gbuf=3)
    se = W.Stream(w, h, pe)
    ost = O.OracleExtStream(w, h, ext_params_from(pe))
    out = torch.empty(3, h, w, device="cuda")
    for f in fr:
        se.denoise(f["radiance"].cuda(), f["motion"].cuda(), out, variance=f["variance"].cuda(),
                   features=f["features"].cuda())
        r = ost.frame(f["radiance"].numpy(), f["motion"].numpy(), f["variance"].numpy(), f["features"].numpy())
        assert rel_err(out.cpu().numpy(), r[0]) <= REL_TOL
    W.wrls_stream_check(se.handle)
    se.close()


def test_missing_samples_and_bad_motion():
    spec = synth.SceneSpec(90, 60, 10, seed=35, motion="orbit", firefly_frac=0.05)

    def hooks(t, rad, mot):
        g = torch.Generator().manual_seed(100 + t)
        m = torch.rand(60, 90, generator=g) < 0.03
        rad[0][m] = float("nan")
        rad[2][torch.rand(60, 90, generator=g) < 0.01] = float("inf")
        mot[0][torch.rand(60, 90, generator=g) < 0.02] = float("nan")
        mot[1][torch.rand(60, 90, generator=g) < 0.02] = 1e6
        mot[0][:, :4] = -7.25                      # leaves the image on the left
        if t == 6:
            rad[:, 10:13, 20:23] = float("nan")    # a 3x3 hole: clamp box of the centre is empty
        return rad, mot
    run_pair(cpu_frames(spec), 90, 60, hooks=hooks)


def test_reset_restarts_every_pixel():
    spec = synth.SceneSpec(64, 40, 8, seed=36, motion="pan", firefly_frac=0.05)
    fr = cpu_frames(spec)
    s = W.Stream(64, 40)
    fresh = W.Stream(64, 40)
    o1 = torch.empty(3, 40, 64, device="cuda")
    o2 = torch.empty_like(o1)
    for t in range(5):
        s.denoise(fr[t]["radiance"].cuda(), fr[t]["motion"].cuda(), o1)
    s.reset()
    s.denoise(fr[5]["radiance"].cuda(), fr[5]["motion"].cuda(), o1)
    fresh.denoise(fr[5]["radiance"].cuda(), fr[5]["motion"].cuda(), o2)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    assert W.wrls_stream_frames(s.handle) == 6


def test_host_entry_matches_device_entry():
    spec = synth.SceneSpec(120, 70, 6, seed=37, motion="orbit", firefly_frac=0.05)
    fr = cpu_frames(spec)
    a = W.Stream(120, 70)
    b = W.Stream(120, 70)
    od = torch.empty(3, 70, 120, device="cuda")
    oh = torch.empty(3, 70, 120).pin_memory()
    for f in fr:
        rad_h, mot_h = f["radiance"].pin_memory(), f["motion"].pin_memory()
        a.denoise(rad_h.cuda(), mot_h.cuda(), od)
        W.wrls_denoise_frame_host(b.handle, rad_h, None, None, mot_h, oh)
        torch.cuda.synchronize()
        assert torch.equal(od.cpu(), oh)


@pytest.mark.parametrize("precision", [W.WRLS_STATE_F32, W.WRLS_STATE_BF16])
def test_batch_tick_equals_each_stream_alone(precision):
    sizes = [(64, 48), (100, 33), (257, 129), (31, 7), (128, 128)]
    specs = [synth.SceneSpec(w, h, 5, seed=40 + i, motion="orbit", firefly_frac=0.05)
             for i, (w, h) in enumerate(sizes)]
    frames = [cpu_frames(sp) for sp in specs]
    p = W.wrls_params_default(state_precision=precision)
    alone = [W.Stream(w, h, p) for (w, h) in sizes]
    mixed = [W.Stream(w, h, p) for (w, h) in sizes]
    batch = W.wrls_batch_create(8)
    try:
        for t in range(5):
            outs_a, outs_b, io = [], [], []
            for i, (w, h) in enumerate(sizes):
                rad, mot = frames[i][t]["radiance"].cuda(), frames[i][t]["motion"].cuda()
                oa = torch.empty(3, h, w, device="cuda")
                ob = torch.empty_like(oa)
                alone[i].denoise(rad, mot, oa)
                io.append((mixed[i].handle, rad, None, None, mot, ob))
                outs_a.append(oa)
                outs_b.append(ob)
            order = [(t + k) % len(sizes) for k in range(len(sizes))]   # any order
            W.wrls_batch_tick(batch, [io[k] for k in order])
            torch.cuda.synchronize()
            for oa, ob in zip(outs_a, outs_b):
                assert torch.equal(oa, ob)
    finally:
        W.wrls_batch_destroy(batch)


def test_full_size_pan_1080p_120_frames():
    """The bench workload at full size (1920x1080, 120 frames, pan 1.7 px/frame, 5% fireflies)
    in the launch configuration bench.py times: one wrls_denoise_sequence call over the 120
    frames on a non-default CUDA stream, default blend configuration, 3 blend CTAs per SM.
    Every pixel of every frame against the oracle; per-frame calls give the same bits."""
    spec = synth.pan_1080p_120f()
    sc = synth.Scene(spec)
    T, H, Wd = spec.frames, spec.height, spec.width
    p = W.wrls_params_default()
    rad = torch.empty(T, 3, H, Wd, device="cuda")
    mot = torch.empty(T, 2, H, Wd, device="cuda")
    for t in range(T):
        f = sc.frame(t)
        rad[t].copy_(f["radiance"])
        mot[t].copy_(f["motion"])
    outs = torch.empty(T, 3, H, Wd, device="cuda")
    seq = W.Stream(Wd, H, p, cuda_stream=torch.cuda.Stream())
    W.wrls_stream_set_overlap(seq.handle, 3)
    W.wrls_denoise_sequence(seq.handle, [(rad[t], None, None, mot[t], outs[t]) for t in range(T)])
    W.wrls_stream_check(seq.handle)  # synchronises the stream's CUDA stream (joined with the blends)
    seq.close()
    pf = W.Stream(Wd, H, p)
    st = O.OracleStream(Wd, H, oracle_params_from(p))
    out = torch.empty(3, H, Wd, device="cuda")
    worst = worst_c = 0.0
    n_c = 0
    for t in range(T):
        pf.denoise(rad[t], mot[t], out)
        torch.cuda.synchronize()
        assert torch.equal(out, outs[t]), t
        ref, _, _ = st.frame(rad[t].cpu().numpy(), mot[t].cpu().numpy())
        o = outs[t].cpu().numpy()
        e = rel_err(o, ref)
        worst = max(worst, e)
        # the per-channel form, reported beside the per-pixel gate
        ec = np.abs(o - ref) / np.maximum(np.abs(ref), FLOOR)
        worst_c = max(worst_c, float(ec.max()))
        n_c += int((ec.max(axis=0) > REL_TOL).sum())
        assert e <= REL_TOL, (t, e)
    W.wrls_stream_check(pf.handle)
    pf.close()
    print("full-size worst rel err: per pixel %.3g; per channel %.3g (%d of %d pixel-frames above %.0e)"
          % (worst, worst_c, n_c, Wd * H * T, REL_TOL))


def test_blend_configs_bitwise_identical_and_autotune():
    spec = synth.SceneSpec(301, 77, 6, seed=50, motion="orbit", firefly_frac=0.05)
    fr = cpu_frames(spec)
    outs = []
    for cfg in range(W.BLEND_CONFIGS):
        s = W.Stream(spec.width, spec.height)
        W.wrls_stream_set_blend_config(s.handle, cfg)
        o = torch.empty(3, spec.height, spec.width, device="cuda")
        for f in fr:
            s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
        torch.cuda.synchronize()
        outs.append(o.clone())
        if cfg == 0:
            times, chosen = W.wrls_stream_autotune(s.handle, o, reps=2)
            assert len(times) == W.BLEND_CONFIGS and all(t > 0 for t in times)
            assert 0 <= chosen < W.BLEND_CONFIGS
            assert torch.equal(o, outs[0])      # the tuner leaves the current output in `out`
        W.wrls_stream_check(s.handle)
        s.close()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("kw", [dict(blend_mode=1), dict(feature_mode=1), dict(radius=1), dict(radius=0)])
def test_blend_configs_bitwise_identical_variants(kw):
    """Every blend configuration (scalar, persistent, two-wide packed) gives the same bits for
    the blend variants too (own predictions, no feature, 3 x 3 window, temporal only), on a
    ragged image, and the two-wide output matches the oracle."""
    spec = synth.SceneSpec(203, 45, 4, seed=52, motion="orbit", firefly_frac=0.05)
    p = W.wrls_params_default(**kw)
    fr = cpu_frames(spec)
    outs = []
    for cfg in range(W.BLEND_CONFIGS):
        s = W.Stream(spec.width, spec.height, p)
        W.wrls_stream_set_blend_config(s.handle, cfg)
        o = torch.empty(3, spec.height, spec.width, device="cuda")
        for f in fr:
            s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
        W.wrls_stream_check(s.handle)
        outs.append(o.cpu())
        s.close()
    for cfg, o in enumerate(outs[1:], 1):
        assert torch.equal(o, outs[0]), cfg
    st = O.OracleStream(spec.width, spec.height, oracle_params_from(p))
    for f in fr:
        ref, _, _ = st.frame(f["radiance"].numpy(), f["motion"].numpy())
    assert rel_err(outs[9].numpy(), ref) <= REL_TOL


@pytest.mark.parametrize("prec", [1, 2])
def test_blend_configs_bitwise_identical_16bit(prec):
    """With BF16 / FP16 state the one-CTA-per-tile blends (0-3) and the two-wide blends (8, 9),
    which copy the 16-bit planes by TMA and decode them in shared memory, give the same bits;
    configurations 4-7 are refused; autotune times 0-3, 8, 9 only."""
    spec = synth.SceneSpec(203, 45, 4, seed=53, motion="orbit", firefly_frac=0.05)
    p = W.wrls_params_default(state_precision=prec)
    fr = cpu_frames(spec)
    outs = {}
    for cfg in (0, 1, 2, 3, 8, 9):
        s = W.Stream(spec.width, spec.height, p)
        W.wrls_stream_set_blend_config(s.handle, cfg)
        o = torch.empty(3, spec.height, spec.width, device="cuda")
        for f in fr:
            s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
        if cfg == 0:
            times, chosen = W.wrls_stream_autotune(s.handle, o, reps=2)
            assert [t > 0 for t in times] == [c in (0, 1, 2, 3, 8, 9) for c in range(W.BLEND_CONFIGS)]
            assert chosen in (0, 1, 2, 3, 8, 9)
            with pytest.raises(W.WrlsError):
                W.wrls_stream_set_blend_config(s.handle, 5)
        W.wrls_stream_check(s.handle)
        outs[cfg] = o.cpu()
        s.close()
    for cfg in (1, 2, 3, 8, 9):
        assert torch.equal(outs[cfg], outs[0]), cfg


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_blend_configs_match_oracle(cfg):
    spec = synth.SceneSpec(197, 53, 5, seed=51, motion="pan", firefly_frac=0.05)
    p = W.wrls_params_default()
    fr = cpu_frames(spec)
    s = W.Stream(spec.width, spec.height, p)
    W.wrls_stream_set_blend_config(s.handle, cfg)
    st = O.OracleStream(spec.width, spec.height, oracle_params_from(p))
    out = torch.empty(3, spec.height, spec.width, device="cuda")
    for f in fr:
        s.denoise(f["radiance"].cuda(), f["motion"].cuda(), out)
        ref, _, _ = st.frame(f["radiance"].numpy(), f["motion"].numpy())
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), ref) <= REL_TOL


@pytest.mark.parametrize("kind", ["uniform", "random"])
def test_staged_and_global_gather_paths(kind):
    """Uniform motion keeps every tile's tap footprint inside the staged window (TMA path);
    per-pixel random motion of a few pixels spreads it beyond (global-gather path)."""
    spec = synth.SceneSpec(160, 96, 8, seed=52, motion="static", firefly_frac=0.05)
    fr = cpu_frames(spec)

    def hooks(t, rad, mot):
        g = torch.Generator().manual_seed(200 + t)
        if kind == "uniform":
            mot[0] = 0.75
            mot[1] = -0.5
        else:
            mot.copy_((torch.rand(2, 96, 160, generator=g) - 0.5) * 12.0)
        return rad, mot
    run_pair(fr, 160, 96, hooks=hooks)


def test_pan_ragged_against_the_oracle():
    spec = synth.SceneSpec(181, 95, 24, seed=56, motion="pan", firefly_frac=0.05)
    run_pair(cpu_frames(spec), spec.width, spec.height)


def test_pipelined_blend_rejected_for_16bit_state():
    s = W.Stream(64, 64, W.wrls_params_default(state_precision=W.WRLS_STATE_BF16))
    with pytest.raises(W.WrlsError):
        W.wrls_stream_set_blend_config(s.handle, 4)
    W.wrls_stream_set_blend_config(s.handle, 3)
    o = torch.empty(3, 64, 64, device="cuda")
    spec = synth.SceneSpec(64, 64, 2, seed=55, motion="orbit")
    for f in cpu_frames(spec):
        s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
    times, chosen = W.wrls_stream_autotune(s.handle, o, reps=1)
    assert all(t < 0 for t in times[4:]) and chosen < 4
    s.close()


def test_bounded_wait_expiry_is_reported_and_the_context_stays_usable():
    """Withhold the state-window copy: each tile's bounded mbarrier wait runs out (about a
    second), the kernel records WRLS_ERR_TIMEOUT and returns; the next frames work."""
    import time
    spec = synth.SceneSpec(64, 48, 4, seed=58, motion="pan", firefly_frac=0.05)
    fr = cpu_frames(spec)
    p = W.wrls_params_default()
    s = W.Stream(64, 48, p)
    st = O.OracleStream(64, 48, oracle_params_from(p))
    o = torch.empty(3, 48, 64, device="cuda")
    s.denoise(fr[0]["radiance"].cuda(), fr[0]["motion"].cuda(), o)   # frame 0 restarts (no copy)
    st.frame(fr[0]["radiance"].numpy(), fr[0]["motion"].numpy())
    W.wrls_stream_check(s.handle)
    W.wrls_stream_set_debug(s.handle, W.WRLS_DEBUG_WITHHOLD_STAGE_COPY)
    t0 = time.time()
    s.denoise(fr[1]["radiance"].cuda(), fr[1]["motion"].cuda(), o)
    with pytest.raises(W.WrlsError) as e:
        W.wrls_stream_check(s.handle)
    assert e.value.status == W.WRLS_ERR_TIMEOUT and time.time() - t0 > 0.3
    W.wrls_stream_set_debug(s.handle, 0)
    s.reset()                                      # the timed-out frame left an unreliable state
    s2 = O.OracleStream(64, 48, oracle_params_from(p))
    for f in fr[2:]:
        s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
        ref, _, _ = s2.frame(f["radiance"].numpy(), f["motion"].numpy())
        torch.cuda.synchronize()
        assert rel_err(o.cpu().numpy(), ref) <= REL_TOL
    W.wrls_stream_check(s.handle)
    s.close()


def test_stream_check_reports_ok():
    spec = synth.SceneSpec(64, 64, 3, seed=53, motion="orbit")
    s = W.Stream(64, 64)
    o = torch.empty(3, 64, 64, device="cuda")
    for f in cpu_frames(spec):
        s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
    W.wrls_stream_check(s.handle)


@pytest.mark.parametrize("precision", [W.WRLS_STATE_BF16, W.WRLS_STATE_F16])
def test_16bit_state_quality_within_one_percent(precision):
    """BF16/FP16 storage of the per-pixel state (P with a per-pixel scale), FP32 compute:
    relMSE of the output against the truth within 1% of the FP32-state path's."""
    spec = synth.SceneSpec(320, 180, 60, seed=54, motion="orbit", firefly_frac=0.05,
                           tf_edit_frame=30, light_move_frame=45)
    fr = cpu_frames(spec)
    res = {}
    for prec in (W.WRLS_STATE_F32, precision):
        p = W.wrls_params_default(state_precision=prec)
        s = W.Stream(spec.width, spec.height, p)
        o = torch.empty(3, spec.height, spec.width, device="cuda")
        errs = []
        for f in fr:
            s.denoise(f["radiance"].cuda(), f["motion"].cuda(), o)
            errs.append(relmse(o.cpu().numpy(), f["truth"].numpy()))
        W.wrls_stream_check(s.handle)
        res[prec] = float(np.mean(errs))
        s.close()
    print("relMSE f32 %.5f  16-bit %.5f" % (res[W.WRLS_STATE_F32], res[precision]))
    assert res[precision] <= 1.01 * res[W.WRLS_STATE_F32]
