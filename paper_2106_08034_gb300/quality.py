"""Quality harness: the paper's ablations and a noise sweep on synthetic sequences, run on
the GPU through the C ABI, scored against the generator's clean truth.

Modes (Sec. 5.3, Fig. 8-9): wRLS vs RLS (w = 1), feature p = [1, z] ("F") vs no feature
p = [1] ("NF"), 5x5 spatio-temporal blend vs temporal-only output; and the alternatives the
paper argues against (Sec. 2.1, 5.2-5.3): an RLS regression on the noisy G-buffers
p = [1, depth, normal] ("RLS-G"), the same G-buffers appended to the paper's predictor
("F+G", d = 8), and the sample-variance weight ("varW"). Scores per sequence:
relMSE = mean((out - I)^2 / (I^2 + 0.01)), PSNR on colours clipped to [0, 1], and temporal
flicker = mean over frames of mean |(out_t - out_{t-1}) - (I_t - I_{t-1})| (the part of the
frame-to-frame change not explained by the truth). The first `skip` frames are excluded.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import torch

from . import synth
from . import wrls as W

MODES = {
    "wRLS-F-5x5": {},
    "RLS-F-5x5": {"weight_mode": 1},
    "wRLS-NF-5x5": {"feature_mode": 1},
    "wRLS-F-temporal": {"radius": 0},
    "RLS-G-5x5": {"weight_mode": 1, "feature_mode": 1, "n_gbuf": 4, "n_features": synth.N_FEATURES},
    "wRLS-F+G-5x5": {"n_gbuf": 4, "n_features": synth.N_FEATURES},
    "varW-F-5x5": {"weight_mode": 2},
}


def score_sequence(spec: synth.SceneSpec, overrides: Optional[dict] = None, device="cuda",
                   skip: int = 4, frames: Optional[list] = None) -> Dict[str, float]:
    p = W.wrls_params_default(**(overrides or {}))
    s = W.Stream(spec.width, spec.height, p)
    sc = synth.Scene(spec)
    out = torch.empty(3, spec.height, spec.width, device=device)
    prev_o = prev_t = None
    rel, mse, flick, n = 0.0, 0.0, 0.0, 0
    rel_in = 0.0
    for t in range(spec.frames):
        f = frames[t] if frames is not None else sc.frame(t, device=device)
        rad, mot, truth = f["radiance"].to(device), f["motion"].to(device), f["truth"].to(device)
        s.denoise(rad, mot, out, variance=f["variance"].to(device), features=f["features"].to(device))
        if t >= skip:
            rel += float(((out - truth) ** 2 / (truth * truth + 1e-2)).mean())
            rel_in += float(((rad - truth) ** 2 / (truth * truth + 1e-2)).mean())
            mse += float(((out.clamp(0, 1) - truth) ** 2).mean())
            if prev_o is not None:
                flick += float(((out - prev_o) - (truth - prev_t)).abs().mean())
            n += 1
        prev_o, prev_t = out.clone(), truth
    W.wrls_stream_check(s.handle)
    s.close()
    mse /= max(n, 1)
    return {"relmse": rel / max(n, 1), "relmse_input": rel_in / max(n, 1),
            "psnr_db": 10 * math.log10(1.0 / max(mse, 1e-12)), "flicker": flick / max(n - 1, 1)}


def ablation_report(spec: synth.SceneSpec, device="cuda") -> Dict[str, Dict[str, float]]:
    frames = [synth.Scene(spec).frame(t, device=device) for t in range(spec.frames)]
    return {name: score_sequence(spec, ov, device, frames=frames) for name, ov in MODES.items()}


def noise_sweep(spec: synth.SceneSpec, mus=(-7.0, -5.5, -4.0, -2.5), device="cuda") -> Dict[float, Dict[str, float]]:
    """Output error against the input noise level (log-variance mean mu), the analogue of
    varying samples per pixel (Sec. 7.4, Fig. 16-17)."""
    import dataclasses
    return {mu: score_sequence(dataclasses.replace(spec, noise_mu=mu), None, device) for mu in mus}


VPT_MODES = {
    "wRLS-F-5x5": {},
    "RLS-F-5x5": {"weight_mode": 1},
    "RLS-G-5x5": {"weight_mode": 1, "feature_mode": 1, "n_gbuf": 4, "n_features": 4},
    "wRLS-F+G-5x5": {"n_gbuf": 4, "n_features": 4},
    "varW-F-5x5": {"weight_mode": 2},
    "wRLS-F-temporal": {"radius": 0},
}


def vpt_ablation(width: int = 320, height: int = 180, frames: int = 24, spp: int = 2, ref_spp: int = 64,
                 seed: int = 12, skip: int = 4, device="cuda") -> Dict[str, Dict[str, float]]:
    """The ablations on path-traced input: every frame of an orbiting camera around the
    procedural volume is rendered at `spp` samples per pixel (wrls_render_vpt), filtered
    (wrls_reconstruct, with the variance output), given velocities from its first-collision
    positions (wrls_velocity_from_world) and denoised; the reference is the same frame at
    `ref_spp` with other random numbers. G-buffer modes regress on the renderer's noisy
    albedo (3 planes) and depth of the closest first collision (Fig. 4). Scores as
    score_sequence, against the reference."""
    ins = []
    for t in range(frames):
        sc = synth.vpt_scene(width, height, t, seed=seed)
        smp = torch.empty(spp, 5, height, width, device=device)
        world = torch.empty(3, height, width, device=device)
        feat = torch.empty(7, height, width, device=device)
        W.wrls_render_vpt(sc, smp, world, feat, frame=t)
        rad = torch.empty(3, height, width, device=device)
        var = torch.empty(height, width, device=device)
        W.wrls_reconstruct(smp, rad, var)
        mot = torch.empty(2, height, width, device=device)
        W.wrls_velocity_from_world(world, synth.orbit_camera(t - 1, width, height), mot)
        ref_sc = dict(sc, seed_hi=sc["seed_hi"] + 0x10000)
        rsmp = torch.empty(ref_spp, 5, height, width, device=device)
        rworld = torch.empty(3, height, width, device=device)
        W.wrls_render_vpt(ref_sc, rsmp, rworld, frame=t)
        ref = torch.empty(3, height, width, device=device)
        W.wrls_reconstruct(rsmp, ref)
        g = torch.stack([feat[4], feat[5], feat[6], feat[0]]).contiguous()   # albedo, depth
        ins.append({"radiance": rad, "variance": var, "motion": mot, "features": g, "truth": ref})
    torch.cuda.synchronize()
    spec = synth.SceneSpec(width, height, frames, seed=seed)
    return {name: score_sequence(spec, ov, device, skip=skip, frames=ins) for name, ov in VPT_MODES.items()}


def edit_recovery(spec: Optional[synth.SceneSpec] = None, device="cuda", window: int = 10,
                  band: float = 1.5) -> Dict[str, object]:
    """Output error around a transfer-function edit and a light move, which the paper handles
    without any reset of the models (Sec. 5.2): relMSE per frame, and per event the mean over
    the `window` frames before it, the peak in the `window` frames after it, the settled level
    (mean over frames t0 + window .. t0 + 2 window - 1) and the number of frames until the error
    is within `band` x the settled level (None if it does not get there within the window)."""
    import dataclasses
    if spec is None:
        spec = dataclasses.replace(synth.orbit_edit_1080p_120f(), width=480, height=272, firefly_frac=0.0)
    p = W.wrls_params_default()
    s = W.Stream(spec.width, spec.height, p)
    sc = synth.Scene(spec)
    out = torch.empty(3, spec.height, spec.width, device=device)
    rel = []
    for t in range(spec.frames):
        f = sc.frame(t, device=device)
        truth = f["truth"].to(device)
        s.denoise(f["radiance"].to(device), f["motion"].to(device), out)
        rel.append(float(((out - truth) ** 2 / (truth * truth + 1e-2)).mean()))
    W.wrls_stream_check(s.handle)
    s.close()
    events = {}
    for name, t0 in (("tf_edit", spec.tf_edit_frame), ("light_move", spec.light_move_frame)):
        if t0 is None or t0 < window or t0 + 2 * window > spec.frames:
            continue
        before = sum(rel[t0 - window:t0]) / window
        settled = sum(rel[t0 + window:t0 + 2 * window]) / window
        back = next((i for i in range(window) if rel[t0 + i] <= band * settled), None)
        events[name] = {"frame": t0, "relmse_before": before, "relmse_peak": max(rel[t0:t0 + window]),
                        "relmse_settled": settled, "frames_to_settle": back}
    return {"relmse_per_frame": rel, "events": events}


def runtime_vs_content(sizes=((960, 540), (1920, 1080)), motions=("static", "pan", "orbit"),
                       seeds=(5, 6), frames: int = 10, skip: int = 3, device="cuda") -> Dict[str, object]:
    """GPU time per frame (update + blend kernels, CUDA events of wrls_stream_enable_timing)
    for sequences of equal size but different content (seeds) and motion, and across sizes:
    the paper states that the cost depends only on the resolution (Sec. 7)."""
    res = {}
    for (w, h) in sizes:
        per = {}
        for m in motions:
            for sd in seeds:
                spec = synth.SceneSpec(w, h, frames, seed=sd, motion=m, firefly_frac=0.05)
                sc = synth.Scene(spec)
                fr = [sc.frame(t, device=device) for t in range(frames)]
                s = W.Stream(w, h, W.wrls_params_default())
                out = torch.empty(3, h, w, device=device)
                for t in range(skip):
                    s.denoise(fr[t]["radiance"], fr[t]["motion"], out)
                W.wrls_stream_enable_timing(s.handle, True)
                for t in range(skip, frames):
                    s.denoise(fr[t]["radiance"], fr[t]["motion"], out)
                u, b, n = W.wrls_stream_kernel_times(s.handle)
                W.wrls_stream_check(s.handle)
                s.close()
                per["%s/%d" % (m, sd)] = (u + b) / n * 1e3
        ts = list(per.values())
        res["%dx%d" % (w, h)] = {"us_per_frame": per, "spread": max(ts) / min(ts),
                                 "ns_per_px": sum(ts) / len(ts) * 1e3 / (w * h)}
    return res
