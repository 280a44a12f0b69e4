"""wrls_denoise_sequence (blend of frame t overlapping the update of frame t+1 on a second
CUDA stream) gives bitwise the outputs of per-frame wrls_denoise_frame calls, and of the
oracle within the parity tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import REL_TOL, cpu_frames, oracle_params_from, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    W.lib()


def _inputs(spec):
    fr = cpu_frames(spec)
    return ([f["radiance"].cuda() for f in fr], [f["motion"].cuda() for f in fr],
            [f["variance"].cuda() for f in fr], [f["features"].cuda() for f in fr], fr)


def _per_frame(spec, p, ins, cfg=None):
    rad, mot, var, feat, _ = ins
    s = W.Stream(spec.width, spec.height, p)
    outs = []
    for t in range(spec.frames):
        o = torch.empty(3, spec.height, spec.width, device="cuda")
        s.denoise(rad[t], mot[t], o, variance=var[t], features=feat[t])
        if t == 0 and cfg is not None:
            W.wrls_stream_set_blend_config(s.handle, cfg)
        outs.append(o)
    torch.cuda.synchronize()
    s.close()
    return [o.cpu() for o in outs]


def _sequence(spec, p, ins, cfg=None, chunk=None, overlap=None, cs=None, debug=0):
    rad, mot, var, feat, _ = ins
    s = W.Stream(spec.width, spec.height, p, cuda_stream=cs)
    if debug:
        W.wrls_stream_set_debug(s.handle, debug)
    if overlap is not None:
        W.wrls_stream_set_overlap(s.handle, overlap)
    outs = [torch.empty(3, spec.height, spec.width, device="cuda") for _ in range(spec.frames)]
    io = [(rad[t], var[t], feat[t], mot[t], outs[t]) for t in range(spec.frames)]
    # frame 0 alone, so that the blend configuration applies from frame 1 as in _per_frame
    W.wrls_denoise_sequence(s.handle, io[:1])
    if cfg is not None:
        W.wrls_stream_set_blend_config(s.handle, cfg)
    step = chunk or spec.frames
    for a in range(1, spec.frames, step):
        W.wrls_denoise_sequence(s.handle, io[a:a + step])
    W.wrls_stream_check(s.handle)  # synchronises the stream's CUDA stream (joined with the blends)
    res = [o.cpu() for o in outs]
    s.close()
    return res


@pytest.mark.parametrize("prec,cfg", [(0, None), (0, 8), (0, 9), (0, 4), (0, 2), (1, None), (1, 9), (2, 2)])
def test_sequence_equals_per_frame(prec, cfg):
    spec = synth.SceneSpec(200, 120, 14, seed=61, motion="orbit", firefly_frac=0.05)
    ins = _inputs(spec)
    p = W.wrls_params_default(state_precision=prec)
    ref = _per_frame(spec, p, ins, cfg)
    for chunk, overlap in ((None, None), (5, 0), (3, 2)):
        got = _sequence(spec, p, ins, cfg, chunk, overlap)
        for t in range(spec.frames):
            assert torch.equal(got[t], ref[t]), (t, chunk, overlap)


@pytest.mark.parametrize("prec", [0, 1])
def test_sequence_with_two_state_copies_equals_per_frame(prec):
    """The sequence entries' fallback when the third state copy cannot be allocated
    (WRLS_DEBUG_NO_THIRD_COPY): the update of frame t+2 then waits for the blend of frame t,
    which reads the copy it overwrites. Outputs are bitwise those of per-frame calls, for the
    device entry (default two-wide blend of a 2^19-pixel image, several chunkings) and the host
    entry."""
    spec = synth.SceneSpec(1024, 520, 9, seed=68, motion="orbit", firefly_frac=0.05)
    ins = _inputs(spec)
    p = W.wrls_params_default(state_precision=prec)
    ref = _per_frame(spec, p, ins)
    for chunk, overlap in ((None, None), (4, 2), (1, None)):
        got = _sequence(spec, p, ins, chunk=chunk, overlap=overlap, debug=W.WRLS_DEBUG_NO_THIRD_COPY)
        for t in range(spec.frames):
            assert torch.equal(got[t], ref[t]), (t, chunk, overlap)
    fr = ins[4]
    pin = [{k: f[k].pin_memory() for k in ("radiance", "motion")} for f in fr]
    got = [torch.full((3, spec.height, spec.width), float("nan")).pin_memory() for _ in fr]
    s = W.Stream(spec.width, spec.height, p)
    W.wrls_stream_set_debug(s.handle, W.WRLS_DEBUG_NO_THIRD_COPY)
    W.wrls_denoise_sequence_host(s.handle, [(pin[t]["radiance"], None, None, pin[t]["motion"], got[t])
                                            for t in range(spec.frames)])
    W.wrls_stream_check(s.handle)
    s.close()
    for t in range(spec.frames):
        assert torch.equal(got[t], ref[t]), t


def test_sequence_extended_path_equals_per_frame():
    spec = synth.SceneSpec(150, 90, 10, seed=62, motion="pan", firefly_frac=0.05)
    ins = _inputs(spec)
    p = W.wrls_params_default(n_features=synth.N_FEATURES, n_gbuf=3, weight_mode=2)
    ref = _per_frame(spec, p, ins)
    got = _sequence(spec, p, ins, chunk=4)
    for t in range(spec.frames):
        assert torch.equal(got[t], ref[t]), t


def test_sequence_matches_oracle_full_hd():
    """1920 x 1080 through the sequence entry on a non-default CUDA stream (the benchmark's
    launch configuration): every pixel of 5 frames within the parity tolerance."""
    spec = synth.SceneSpec(1920, 1080, 5, seed=63, motion="pan", firefly_frac=0.05)
    ins = _inputs(spec)
    p = W.wrls_params_default()
    got = _sequence(spec, p, ins, cfg=8, cs=torch.cuda.Stream())
    st = O.OracleStream(spec.width, spec.height, oracle_params_from(p))
    for t, f in enumerate(ins[4]):
        ref, _, _ = st.frame(f["radiance"].numpy(), f["motion"].numpy())
        assert rel_err(got[t].numpy(), ref) <= REL_TOL, t


def test_sequence_kernel_timing_and_rejections():
    spec = synth.SceneSpec(128, 64, 6, seed=64, motion="pan")
    rad, mot, var, feat, _ = _inputs(spec)
    s = W.Stream(spec.width, spec.height)
    W.wrls_stream_enable_timing(s.handle, True)
    outs = [torch.empty(3, spec.height, spec.width, device="cuda") for _ in range(spec.frames)]
    W.wrls_denoise_sequence(s.handle, [(rad[t], None, None, mot[t], outs[t]) for t in range(spec.frames)])
    u, b, n = W.wrls_stream_kernel_times(s.handle)
    assert n == spec.frames and u > 0 and b > 0
    # the output of frame i may not overlap a buffer of frame i+1
    with pytest.raises(W.WrlsError) as e:
        W.wrls_denoise_sequence(s.handle, [(rad[0], None, None, mot[0], outs[0]),
                                           (rad[1], None, None, mot[1], outs[0])])
    assert e.value.status == W.WRLS_ERR_INVALID_ARG
    with pytest.raises(W.WrlsError):
        W.wrls_denoise_sequence(s.handle, [])
    with pytest.raises(W.WrlsError):
        W.wrls_stream_set_overlap(s.handle, -1)
    other = W.Stream(spec.width, spec.height)
    arr = (W.wrls_frame_io * 1)()
    arr[0] = W.wrls_frame_io(other.handle, rad[0].data_ptr(), None, None, mot[0].data_ptr(), outs[0].data_ptr())
    assert W.lib().wrls_denoise_sequence(s.handle, arr, 1) == W.WRLS_ERR_INVALID_ARG
    W.wrls_stream_check(s.handle)
    other.close()
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_sequence_and_per_frame_calls_interleave(prec):
    """Sequence calls (which add a third state copy to the rotation on their first use) and
    per-frame calls on one stream give the per-frame results bit for bit, and the state read
    back at the end is the same."""
    spec = synth.SceneSpec(120, 72, 14, seed=65, motion="orbit", firefly_frac=0.05)
    ins = _inputs(spec)
    rad, mot, var, feat, _ = ins
    p = W.wrls_params_default(state_precision=prec)
    ref = _per_frame(spec, p, ins)
    s = W.Stream(spec.width, spec.height, p)
    outs = [torch.empty(3, spec.height, spec.width, device="cuda") for _ in range(spec.frames)]
    io = [(rad[t], None, None, mot[t], outs[t]) for t in range(spec.frames)]
    W.wrls_denoise_sequence(s.handle, io[0:5])
    for t in range(5, 8):
        s.denoise(rad[t], mot[t], outs[t])
    W.wrls_denoise_sequence(s.handle, io[8:12])
    for t in range(12, 14):
        s.denoise(rad[t], mot[t], outs[t])
    st_a = torch.empty(25, spec.height, spec.width, device="cuda")
    s.read_state(st_a)
    W.wrls_stream_check(s.handle)
    for t in range(spec.frames):
        assert torch.equal(outs[t].cpu(), ref[t]), t
    s2 = W.Stream(spec.width, spec.height, p)
    for t in range(spec.frames):
        s2.denoise(rad[t], mot[t], outs[0])
    st_b = torch.empty_like(st_a)
    s2.read_state(st_b)
    torch.cuda.synchronize()
    assert torch.equal(st_a, st_b)
    s.close()
    s2.close()


@pytest.mark.parametrize("kw,chunks", [(dict(), (5, 9)), (dict(state_precision=1), (14,)),
                                       (dict(n_features=synth.N_FEATURES, n_gbuf=2, weight_mode=2), (4, 10))])
def test_host_sequence_equals_per_frame_host_calls(kw, chunks):
    """wrls_denoise_sequence_host (input copies, kernels and output copies of consecutive
    frames overlapping on three streams, three device slots reused) gives bit for bit the
    outputs of per-frame host calls, including across calls and slot reuse."""
    spec = synth.SceneSpec(160, 96, 14, seed=66, motion="orbit", firefly_frac=0.05)
    fr = cpu_frames(spec)
    p = W.wrls_params_default(**kw)
    pin = [{k: f[k].pin_memory() for k in ("radiance", "motion", "variance", "features")} for f in fr]
    ref = [torch.empty(3, spec.height, spec.width).pin_memory() for _ in fr]
    s = W.Stream(spec.width, spec.height, p)
    for t, f in enumerate(pin):
        W.wrls_denoise_frame_host(s.handle, f["radiance"], f["variance"], f["features"], f["motion"], ref[t])
    W.wrls_stream_check(s.handle)
    s.close()
    got = [torch.full((3, spec.height, spec.width), float("nan")).pin_memory() for _ in fr]
    s = W.Stream(spec.width, spec.height, p)
    a = 0
    for c in chunks:
        W.wrls_denoise_sequence_host(s.handle, [(pin[t]["radiance"], pin[t]["variance"], pin[t]["features"],
                                                 pin[t]["motion"], got[t]) for t in range(a, a + c)])
        a += c
    W.wrls_stream_check(s.handle)   # synchronises the stream's CUDA stream, joined with the copies
    s.close()
    for t in range(spec.frames):
        assert torch.equal(got[t], ref[t]), t


@pytest.mark.parametrize("kw", [dict(), dict(state_precision=1), dict(n_features=synth.N_FEATURES, n_gbuf=2, weight_mode=2)])
def test_state_checkpoint_resume(kw):
    """wrls_stream_read_state of stream A loaded into a fresh stream B with
    wrls_stream_write_state resumes A: with the binary32 state B's next frames equal A's bit for
    bit (also on the extended path); with BF16 they agree within the parity tolerance."""
    spec = synth.SceneSpec(150, 84, 12, seed=67, motion="orbit", firefly_frac=0.05)
    fr = cpu_frames(spec)
    p = W.wrls_params_default(**kw)
    a = W.Stream(spec.width, spec.height, p)
    b = W.Stream(spec.width, spec.height, p)
    out = torch.empty(3, spec.height, spec.width, device="cuda")
    ins = [(f["radiance"].cuda(), f["motion"].cuda(), f["variance"].cuda(), f["features"].cuda()) for f in fr]
    for t in range(6):
        a.denoise(ins[t][0], ins[t][1], out, variance=ins[t][2], features=ins[t][3])
    npl = a.state_planes
    st = torch.empty(npl, spec.height, spec.width, device="cuda")
    a.read_state(st)
    b.write_state(st)
    st_b = torch.empty_like(st)
    b.read_state(st_b)
    if kw.get("state_precision", 0) == 0:
        assert torch.equal(st_b, st)
    oa = torch.empty_like(out)
    ob = torch.empty_like(out)
    for t in range(6, spec.frames):
        a.denoise(ins[t][0], ins[t][1], oa, variance=ins[t][2], features=ins[t][3])
        b.denoise(ins[t][0], ins[t][1], ob, variance=ins[t][2], features=ins[t][3])
        if kw.get("state_precision", 0) == 0:
            assert torch.equal(oa, ob), t
        else:
            assert rel_err(ob.cpu().numpy(), oa.cpu().numpy()) <= REL_TOL * 10, t
    W.wrls_stream_check(a.handle)
    W.wrls_stream_check(b.handle)
    assert W.lib().wrls_stream_write_state(None, st.data_ptr()) == W.WRLS_ERR_INVALID_ARG
    a.close()
    b.close()


@pytest.mark.parametrize("kw", [dict(), dict(state_precision=1), dict(feature_mode=1),
                                dict(n_features=synth.N_FEATURES, n_gbuf=2, weight_mode=2),
                                dict(p_trace_max=3.0)])
def test_state_stats_match_the_state(kw):
    """wrls_stream_state_stats agrees with the state read back: trace(P) max and mean and the
    smallest diagonal over the used block, no non-finite values; with the reset guard on,
    trace(P) never exceeds max(p_trace_max, trace(P0))."""
    spec = synth.SceneSpec(141, 77, 9, seed=68, motion="orbit", firefly_frac=0.05)
    fr = cpu_frames(spec)
    p = W.wrls_params_default(**kw)
    s = W.Stream(spec.width, spec.height, p)
    with pytest.raises(W.WrlsError):
        W.wrls_stream_state_stats(s.handle)          # no frame yet
    out = torch.empty(3, spec.height, spec.width, device="cuda")
    for f in fr:
        s.denoise(f["radiance"].cuda(), f["motion"].cuda(), out, variance=f["variance"].cuda(),
                  features=f["features"].cuda())
    st = W.wrls_stream_state_stats(s.handle)
    planes = torch.empty(s.state_planes, spec.height, spec.width, device="cuda")
    s.read_state(planes)
    pl = planes.double().cpu()
    if "n_gbuf" in kw:
        d = int(round((-7 + (49 + 8 * (s.state_planes - 3)) ** 0.5) / 2))  # 3d + d(d+1)/2 + 3 planes
        idx, e = [], 3 * d
        for a in range(d):
            idx.append(e)
            e += d - a
    else:
        idx = [12] if kw.get("feature_mode", 0) == 1 else [12, 16, 19, 21]
    diag = pl[idx]
    tr = diag.sum(0)
    assert st["frames"] == spec.frames and st["nonfinite"] == 0
    assert st["p_trace_max"] == pytest.approx(float(tr.max()), rel=1e-5)
    assert st["p_trace_mean"] == pytest.approx(float(tr.mean()), rel=1e-5)
    assert st["p_diag_min"] == pytest.approx(float(diag.min()), rel=1e-5) and st["p_diag_min"] > 0
    if "p_trace_max" in kw:
        assert st["p_trace_max"] <= max(kw["p_trace_max"], 4 * p.p0_delta) * (1 + 1e-6)
    W.wrls_stream_check(s.handle)
    s.close()
