"""State-format precision of the CUDA path against the FP64 oracle (Sec. 5.2, Eq. 10-11, 14:
the recursion that the stored state carries from frame to frame).

- A gate that can fail: on a firefly-free orbit sequence with a transfer-function edit and a
  light move, the relMSE against the truth of the BF16 / FP16 state paths stays within 1 % of
  the binary32 path's, and their error against the oracle stays within the bounds stated here.
- Long runs: 1200 frames (more than twice the effective memory 1/(1 - lambda) = 500 frames
  of lambda = 0.998) at 128 x 128, static camera and pan, 5 % fireflies: the binary32 state
  still meets the parity bound on every frame, and trace(P) read back from the device follows
  the oracle's; the BF16 and FP16 states' errors stay within the bounds stated here (the
  Cholesky-factor storage of P keeps the decoded P positive semi-definite; an entry-by-entry
  16-bit P diverged on this sequence).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import FLOOR, REL_TOL, cpu_frames, oracle_params_from, rel_err, rel_err_channel, relmse

pytestmark = pytest.mark.gpu

# Bounds of the 16-bit state formats against the oracle (per-pixel metric of the parity gate,
# helpers.rel_err) on the 120-frame orbit sequences below: the mean over pixels and frames,
# and the worst pixel, at about twice the measured values (BF16: mean 1.3e-3 / 1.5e-3, worst
# 0.044 / 0.10 without / with the edits; FP16: mean 1.5e-4, worst 0.0066). BF16 keeps 8
# significant bits (relative rounding 2^-9), FP16 11. The worst pixels are fireflies' neighbours,
# where the cross prediction p_i . beta_k multiplies the neighbours' rounded beta by |z_i| >> 1.
BOUND_16 = {W.WRLS_STATE_BF16: {"mean": 3e-3, "max": 0.25}, W.WRLS_STATE_F16: {"mean": 4e-4, "max": 0.02}}
# The same with 5 % fireflies (x50), on the 16-stream mix at full size over its first 3 frames:
# the mean, the 99.9th percentile and the worst pixel at about twice the measured values (BF16:
# mean 9.4e-4, p99.9 6.6e-3, worst 1.28; FP16: 1.2e-4, 8.2e-4, 0.157). A firefly's sample enters its
# pixel's feature through Eq. 12, |z_i| >> 1, and the cross prediction multiplies the
# neighbours' rounded beta by it; where the oracle's colour at such a pixel is small, the
# per-pixel error is large while 999 pixels in 1000 stay below 1e-2.
BOUND_16_FIREFLIES = {W.WRLS_STATE_BF16: {"mean": 2e-3, "p999": 1.5e-2, "max": 2.6},
                      W.WRLS_STATE_F16: {"mean": 2.5e-4, "p999": 1.7e-3, "max": 0.32}}
# Long histories (1200 frames at 128 x 128, 5 % fireflies): bounds of the mean error of each
# 100-frame block and of the worst pixel, at about twice the measured static-camera values
# (BF16: block mean rising to 3.7e-2, worst 5.3; FP16: 2.8e-3, worst 0.54). The 16-bit states
# lag the binary32 one more the longer a pixel's history: a frame changes the state by about
# (1 - lambda) = 0.2 % relative, less than BF16's rounding step (0.4 %) and a few of FP16's
# steps, so part of each update rounds away.
# relMSE against the truth over the last 300 frames within 1 % above the binary32 path's (measured
# ratios: BF16 0.985 / 1.000 / 0.887, FP16 0.999 / 1.000 / 1.000 for static / pan / static without
# fireflies; BF16's is lower on long static runs, where its rounded slopes of beta stay smaller).
LONG_16 = {W.WRLS_STATE_BF16: {"mean": 0.08, "max": 12.0, "relmse_ratio": 1.01},
           W.WRLS_STATE_F16: {"mean": 6e-3, "max": 1.5, "relmse_ratio": 1.01}}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    W.lib()


def per_pixel_err(gpu, ref):
    """Per-pixel relative error field (H, W) of the parity metric."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.max(np.abs(gpu - ref), axis=0) / np.maximum(np.max(np.abs(ref), axis=0), FLOOR)


@pytest.mark.parametrize("edits", [False, True])
@pytest.mark.parametrize("precision", [W.WRLS_STATE_BF16, W.WRLS_STATE_F16])
def test_16bit_state_gate_without_fireflies(precision, edits):
    """320x180, 120 frames, orbit, no fireflies (relMSE ~ 1e-2, so that 1 % of it is a real
    bound); with `edits`, a transfer-function edit at frame 60 and a light move at frame 90."""
    spec = synth.SceneSpec(320, 180, 120, seed=81, motion="orbit", firefly_frac=0.0,
                           tf_edit_frame=60 if edits else None, light_move_frame=90 if edits else None)
    fr = cpu_frames(spec)
    st = O.OracleStream(spec.width, spec.height, oracle_params_from(W.wrls_params_default()))
    streams = {p: W.Stream(spec.width, spec.height, W.wrls_params_default(state_precision=p))
               for p in (W.WRLS_STATE_F32, precision)}
    outs = {p: torch.empty(3, spec.height, spec.width, device="cuda") for p in streams}
    rm = {p: [] for p in streams}
    errs = {p: [] for p in streams}
    for f in fr:
        for p, s in streams.items():
            s.denoise(f["radiance"].cuda(), f["motion"].cuda(), outs[p])
        ref, _, _ = st.frame(f["radiance"].numpy(), f["motion"].numpy())
        for p in streams:
            o = outs[p].cpu().numpy()
            rm[p].append(relmse(o, f["truth"].numpy()))
            errs[p].append(per_pixel_err(o, ref))
    for s in streams.values():
        W.wrls_stream_check(s.handle)
        s.close()
    r32, r16 = float(np.mean(rm[W.WRLS_STATE_F32])), float(np.mean(rm[precision]))
    e16 = np.stack(errs[precision])
    print("relMSE f32 %.6f  16-bit %.6f  ratio %.5f;  16-bit vs oracle: mean %.3g  p99.9 %.3g  max %.3g;"
          "  f32 vs oracle max %.3g" % (r32, r16, r16 / r32, e16.mean(), np.quantile(e16, 0.999), e16.max(),
                                        np.max(errs[W.WRLS_STATE_F32])))
    assert 0.003 < r32 < (0.3 if edits else 0.03), "the firefly-free relMSE is what makes the 1 % gate sensitive"
    assert r16 <= 1.01 * r32
    assert np.max(errs[W.WRLS_STATE_F32]) <= REL_TOL
    assert e16.mean() <= BOUND_16[precision]["mean"]
    assert e16.max() <= BOUND_16[precision]["max"]


@pytest.mark.parametrize("precision", [W.WRLS_STATE_F32, W.WRLS_STATE_BF16, W.WRLS_STATE_F16])
def test_batched_mix_full_size_against_the_oracle(precision):
    """The batched workload at full size: the 16 streams of the mix (4 x 512^2, 4 x 1280x720,
    4 x 1920x1080, 2 x 2560x1440, 2 x 3840x2160; orbit, 5 % fireflies, independent seeds),
    3 ticks through wrls_batch_tick with each stream at its default blend configuration (the
    two-wide TMA blends on the large streams). The outputs equal each stream's per-frame calls
    bit for bit, and against the oracle (every pixel of every frame) the binary32 state meets
    the parity bound and the 16-bit states the bounds stated above for sequences with fireflies."""
    specs = synth.mix16_60f(frames=3)
    p = W.wrls_params_default(state_precision=precision)
    scenes = [synth.Scene(sp) for sp in specs]
    alone = [W.Stream(sp.width, sp.height, p) for sp in specs]
    mixed = [W.Stream(sp.width, sp.height, p) for sp in specs]
    inputs = [[] for _ in specs]   # (radiance, motion, batched output) per frame, on the device
    batch = W.wrls_batch_create(len(specs))
    try:
        for t in range(3):
            io, pairs = [], []
            for i, sp in enumerate(specs):
                f = scenes[i].frame(t, device="cuda")
                oa = torch.empty(3, sp.height, sp.width, device="cuda")
                ob = torch.empty_like(oa)
                alone[i].denoise(f["radiance"], f["motion"], oa)
                io.append((mixed[i].handle, f["radiance"], None, None, f["motion"], ob))
                pairs.append((oa, ob))
                inputs[i].append((f["radiance"], f["motion"], ob))
            W.wrls_batch_tick(batch, io[::-1])   # any order
            torch.cuda.synchronize()
            for i, (oa, ob) in enumerate(pairs):
                assert torch.equal(oa, ob), (t, i)
    finally:
        W.wrls_batch_destroy(batch)
    for s in alone + mixed:
        W.wrls_stream_check(s.handle)
        s.close()
    errs = []
    for i, sp in enumerate(specs):   # one oracle stream at a time (FP64 state of a 4K stream: 3.3 GB)
        st = O.OracleStream(sp.width, sp.height, oracle_params_from(W.wrls_params_default()))
        for rad, mot, ob in inputs[i]:
            ref, _, _ = st.frame(rad.cpu().numpy(), mot.cpu().numpy())
            errs.append(per_pixel_err(ob.cpu().numpy(), ref).ravel())
        del st
    e = np.concatenate(errs)
    print("mix16 full size, 3 ticks, state %d: vs oracle mean %.3g  p99.9 %.3g  max %.3g"
          % (precision, e.mean(), np.quantile(e, 0.999), e.max()))
    if precision == W.WRLS_STATE_F32:
        assert e.max() <= REL_TOL
    else:
        b = BOUND_16_FIREFLIES[precision]
        assert e.mean() <= b["mean"]
        assert np.quantile(e, 0.999) <= b["p999"]
        assert e.max() <= b["max"]


def test_orbit_edit_1080p_120_frames_every_format():
    """The precision workload at full size (1920x1080, 120 frames, orbit, 5 % fireflies,
    transfer-function edit at frame 60, light move at frame 90): every pixel of every frame of
    the binary32, BF16 and FP16 state paths against the oracle, on the same inputs. The binary32
    state meets the parity bound; the 16-bit states the bounds stated above for sequences with
    fireflies (the 99.9th percentile as a count of pixel-frames above it)."""
    spec = synth.orbit_edit_1080p_120f()
    sc = synth.Scene(spec)
    fmts = (W.WRLS_STATE_F32, W.WRLS_STATE_BF16, W.WRLS_STATE_F16)
    streams = {p: W.Stream(spec.width, spec.height, W.wrls_params_default(state_precision=p)) for p in fmts}
    outs = {p: torch.empty(3, spec.height, spec.width, device="cuda") for p in fmts}
    st = O.OracleStream(spec.width, spec.height, oracle_params_from(W.wrls_params_default()))
    worst = {p: 0.0 for p in fmts}
    total = {p: 0.0 for p in fmts}
    above = {p: 0 for p in fmts}
    for t in range(spec.frames):
        f = sc.frame(t, device="cuda")
        for p in fmts:
            streams[p].denoise(f["radiance"], f["motion"], outs[p])
        ref, _, _ = st.frame(f["radiance"].cpu().numpy(), f["motion"].cpu().numpy())
        for p in fmts:
            e = per_pixel_err(outs[p].cpu().numpy(), ref)
            worst[p] = max(worst[p], float(e.max()))
            total[p] += float(e.sum())
            if p != W.WRLS_STATE_F32:
                above[p] += int((e > BOUND_16_FIREFLIES[p]["p999"]).sum())
    for s in streams.values():
        W.wrls_stream_check(s.handle)
        s.close()
    n = spec.width * spec.height * spec.frames
    print("orbit/edit 1080p x 120: " + "; ".join(
        "state %d max %.3g mean %.3g" % (p, worst[p], total[p] / n) for p in fmts))
    assert worst[W.WRLS_STATE_F32] <= REL_TOL
    for p in fmts[1:]:
        b = BOUND_16_FIREFLIES[p]
        assert total[p] / n <= b["mean"], p
        assert above[p] <= 0.001 * n, p
        assert worst[p] <= b["max"], p


@pytest.mark.parametrize("motion,fireflies", [("static", 0.05), ("pan", 0.05), ("static", 0.0)])
def test_long_run_against_the_oracle(motion, fireflies):
    """1200 frames at 128 x 128 with 5 % x50 fireflies (and a firefly-free static run, where the
    relMSE comparison with the truth is sensitive). Binary32 state: within the parity bound
    on every frame, trace(P) on the device within 1e-3 of the oracle's. 16-bit states: bounded
    (the static camera is their worst case: every frame changes the state by about 1 - lambda
    relative, below the 16-bit rounding step). Prints the worst and mean error of each
    100-frame block."""
    T = 1200
    spec = synth.SceneSpec(128, 128, 8, seed=82, motion=motion, firefly_frac=fireflies)
    sc = synth.Scene(spec)
    p32 = W.wrls_params_default()
    st = O.OracleStream(128, 128, oracle_params_from(p32))
    precs = (W.WRLS_STATE_F32, W.WRLS_STATE_BF16, W.WRLS_STATE_F16)
    streams = {p: W.Stream(128, 128, W.wrls_params_default(state_precision=p)) for p in precs}
    outs = {p: torch.empty(3, 128, 128, device="cuda") for p in precs}
    worst = {p: [] for p in precs}
    means = {p: [] for p in precs}
    wc, traces = [], []
    bw = {p: 0.0 for p in precs}
    bs = {p: 0.0 for p in precs}
    rm = {p: [] for p in precs}         # relMSE against the truth over the last 300 frames
    bwc = 0.0
    for t in range(T):
        f = sc.frame(t)
        for p in precs:
            streams[p].denoise(f["radiance"].cuda(), f["motion"].cuda(), outs[p])
        ref, _, _ = st.frame(f["radiance"].numpy(), f["motion"].numpy())
        for p in precs:
            o = outs[p].cpu().numpy()
            e = per_pixel_err(o, ref)
            bw[p] = max(bw[p], float(e.max()))
            bs[p] += float(e.mean())
            if t >= T - 300:
                rm[p].append(relmse(o, f["truth"].numpy()))
        bwc = max(bwc, rel_err_channel(outs[W.WRLS_STATE_F32].cpu().numpy(), ref))
        e32 = rel_err(outs[W.WRLS_STATE_F32].cpu().numpy(), ref)
        assert e32 <= REL_TOL, "frame %d: binary32 state error %.3g" % (t, e32)
        if (t + 1) % 100 == 0:
            g = W.wrls_stream_state_stats(streams[W.WRLS_STATE_F32].handle)
            tr = np.trace(st.P, axis1=1, axis2=2)
            traces.append((t + 1, g["p_trace_max"], float(tr.max())))
            assert abs(g["p_trace_max"] - tr.max()) <= 1e-3 * tr.max()
            assert g["nonfinite"] == 0
            for p in precs:
                worst[p].append(bw[p])
                means[p].append(bs[p] / 100)
                bw[p], bs[p] = 0.0, 0.0
            wc.append(bwc)
            bwc = 0.0
    for s in streams.values():
        W.wrls_stream_check(s.handle)
        s.close()
    names = {W.WRLS_STATE_F32: "f32", W.WRLS_STATE_BF16: "bf16", W.WRLS_STATE_F16: "f16"}
    r = {p: float(np.mean(rm[p])) for p in precs}
    print("%s, fireflies %.2f, per 100 frames: %s; f32 per-channel worst %s; trace(P) max device/oracle %s; "
          "relMSE vs truth (last 300 frames) %s" % (
              motion, fireflies, "; ".join("%s worst %s mean %s" % (names[p], " ".join("%.2e" % e for e in worst[p]),
                                                        " ".join("%.2e" % e for e in means[p])) for p in precs),
              " ".join("%.2e" % e for e in wc), ["%d: %.4g/%.4g" % x for x in traces],
              ", ".join("%s %.6f (x%.4f)" % (names[p], r[p], r[p] / r[W.WRLS_STATE_F32]) for p in precs)))
    for p in (W.WRLS_STATE_BF16, W.WRLS_STATE_F16):
        assert max(means[p]) <= LONG_16[p]["mean"], (names[p], means[p])
        assert max(worst[p]) <= LONG_16[p]["max"], (names[p], worst[p])
        assert r[p] <= LONG_16[p]["relmse_ratio"] * r[W.WRLS_STATE_F32], (names[p], r)


@pytest.mark.parametrize("precision", [W.WRLS_STATE_BF16, W.WRLS_STATE_F16])
def test_16bit_p_encoding_round_trip(precision):
    """The 16-bit formats store P as the Cholesky factor of P / s, s a power of two: a state
    written with wrls_stream_write_state and read back gives P within a few rounding steps of
    the format relative to max diag P, positive semi-definite, over scales 1e-30 .. 1e30,
    eigenvalue spreads up to 1e6, singular P (one predictor entry unused) and P = p0 I; beta and
    z come back rounded to the format; a non-finite P stays non-finite (counted by the stats)."""
    rng = np.random.default_rng(90)
    Wd, Hd = 64, 32
    n = Wd * Hd
    st = np.zeros((25, n))
    st[0:12] = rng.normal(0, 2, (12, n))
    st[22:25] = rng.uniform(-3, 3, (3, n))
    Ps = []
    for j in range(n):
        kind = j % 6
        if kind == 5:
            P = np.eye(4)                                    # a restarted pixel
        else:
            Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
            ev = 10.0 ** rng.uniform(-6 if kind < 3 else -2, 0, 4)
            if kind == 4:
                ev[3] = 0.0                                  # singular
            P = (Q * ev) @ Q.T
        P = P * 10.0 ** rng.uniform(-30, 30) if kind == 3 else P * 10.0 ** rng.uniform(-4, 4)
        Ps.append(P)
    iu = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
    for q, (a, b) in enumerate(iu):
        st[12 + q] = [P[a, b] for P in Ps]
    src = torch.from_numpy(st.reshape(25, Hd, Wd).astype(np.float32)).cuda()
    s = W.Stream(Wd, Hd, W.wrls_params_default(state_precision=precision))
    s.write_state(src)
    back = torch.empty_like(src)
    s.read_state(back)
    torch.cuda.synchronize()
    got = back.double().cpu().numpy().reshape(25, n)
    ref = src.double().cpu().numpy().reshape(25, n)   # the binary32 values that were written
    step = 2.0 ** -8 if precision == W.WRLS_STATE_BF16 else 2.0 ** -11   # one rounding step
    tiny = 0.0 if precision == W.WRLS_STATE_BF16 else 2.0 ** -25          # half FP16 subnormal step
    assert np.all(np.abs(got[0:12] - ref[0:12]) <= step * np.abs(ref[0:12]) + tiny)
    assert np.all(np.abs(got[22:25] - ref[22:25]) <= step * np.abs(ref[22:25]) + tiny)
    worst = 0.0
    for j in range(n):
        Pg = np.zeros((4, 4))
        Pr = np.zeros((4, 4))
        for q, (a, b) in enumerate(iu):
            Pg[a, b] = Pg[b, a] = got[12 + q, j]
            Pr[a, b] = Pr[b, a] = ref[12 + q, j]
        m = np.max(np.diag(Pr))
        worst = max(worst, np.max(np.abs(Pg - Pr)) / m)
        assert np.min(np.linalg.eigvalsh(Pg)) >= -1e-6 * m, j     # positive semi-definite
    print("worst |dP| / max diag P: %.3g (%.1f rounding steps)" % (worst, worst / step))
    assert worst <= 8 * step
    # a non-finite P entry stays non-finite and is counted
    st[12 + 1, 0] = np.nan
    s.write_state(torch.from_numpy(st.reshape(25, Hd, Wd).astype(np.float32)).cuda())
    assert W.wrls_stream_state_stats(s.handle)["nonfinite"] > 0
    s.close()


@pytest.mark.parametrize("precision", [W.WRLS_STATE_BF16, W.WRLS_STATE_F16])
@pytest.mark.parametrize("wh,kind", [((160, 96), "random"), ((33, 9), "orbit"), ((1, 37), "orbit")])
def test_16bit_global_gather_and_small_images(precision, wh, kind):
    """The 16-bit state where the update reads its taps from global memory (per-pixel random
    motion of a few pixels spreads a tile's taps beyond the staged window; images smaller than
    the window have none): finite outputs within the format's stated mean error of the binary32
    path, and the sequence entry bitwise equal to per-frame calls."""
    w, h = wh
    spec = synth.SceneSpec(w, h, 8, seed=91, motion="static" if kind == "random" else "orbit",
                           firefly_frac=0.05)
    fr = cpu_frames(spec)
    if kind == "random":
        for t, f in enumerate(fr):
            g = torch.Generator().manual_seed(300 + t)
            f["motion"] = (torch.rand(2, h, w, generator=g) - 0.5) * 12.0
    ins = [(f["radiance"].cuda(), f["motion"].cuda()) for f in fr]
    s32 = W.Stream(w, h)
    s16 = W.Stream(w, h, W.wrls_params_default(state_precision=precision))
    o32 = torch.empty(3, h, w, device="cuda")
    per = []
    errs = []
    for rad, mot in ins:
        s32.denoise(rad, mot, o32)
        o16 = torch.empty(3, h, w, device="cuda")
        s16.denoise(rad, mot, o16)
        per.append(o16)
        errs.append(per_pixel_err(o16.cpu().numpy(), o32.cpu().numpy()))
    for s in (s32, s16):
        W.wrls_stream_check(s.handle)
        s.close()
    assert all(torch.isfinite(o).all() for o in per)
    e = np.stack(errs)
    print("%s %dx%d %s: mean %.3g max %.3g vs binary32" % ("bf16" if precision == 1 else "f16", w, h, kind,
                                                            e.mean(), e.max()))
    assert e.mean() <= BOUND_16[precision]["mean"]
    sq = W.Stream(w, h, W.wrls_params_default(state_precision=precision))
    seq = [torch.empty(3, h, w, device="cuda") for _ in ins]
    W.wrls_denoise_sequence(sq.handle, [(rad, None, None, mot, seq[t]) for t, (rad, mot) in enumerate(ins)])
    W.wrls_stream_check(sq.handle)
    sq.close()
    for a, b in zip(per, seq):
        assert torch.equal(a, b)
