"""The CUDA path tracer (wrls_render_vpt) against the FP64 oracle (oracle/wrls_oracle_vpt.c).

Both draw the same Philox4x32-10 numbers, so almost every path is the same path; a path can
still branch differently where a binary32 and a binary64 value fall on opposite sides of a
random threshold (delta tracking's acceptance test, a box exit), after which it is another
valid path. Hence: the sub-pixel offsets are compared bit for bit, the exact physics (a
white furnace) sample for sample, the sample colours by the fraction that agree to 1e-3
(>= 99.5 %), the image means within 5 standard errors, and the transmittance against its
closed form."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import FLOOR, REL_TOL, oracle_params_from, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    W.lib()


def _render_gpu(sc, Wd, Hd, spp, frame=0):
    smp = torch.empty(spp, 5, Hd, Wd, device="cuda")
    world = torch.empty(3, Hd, Wd, device="cuda")
    feat = torch.empty(7, Hd, Wd, device="cuda")
    W.wrls_render_vpt(sc, smp, world, feat, frame=frame)
    torch.cuda.synchronize()
    return smp.cpu().numpy(), world.cpu().numpy(), feat.cpu().numpy()


def _sample_agreement(a, b):
    """Fraction of samples whose colour vectors agree to REL_TOL (relative, floor FLOOR)."""
    num = np.abs(a[:, :3].astype(np.float64) - b[:, :3]).max(1)
    den = np.maximum(np.abs(b[:, :3].astype(np.float64)).max(1), FLOOR)
    return float((num / den <= REL_TOL).mean())


@pytest.mark.parametrize("frame,size", [(0, (96, 64)), (3, (131, 77))])
def test_samples_match_the_oracle(frame, size):
    Wd, Hd = size
    sc = synth.vpt_scene(Wd, Hd, frame, seed=2)
    g_smp, g_world, g_feat = _render_gpu(sc, Wd, Hd, 2, frame)
    o_smp, o_world, o_feat = O.render_vpt(sc, Wd, Hd, 2, frame=frame)
    assert np.array_equal(g_smp[:, 3:], o_smp[:, 3:])             # offsets: bit for bit
    agree = _sample_agreement(g_smp, o_smp)
    assert agree >= 0.995, agree
    n = g_smp[:, :3].size
    for c in range(3):
        # 5 standard errors of the paths that branched, plus binary32 rounding of the rest
        diff = g_smp[:, c].astype(np.float64) - o_smp[:, c]
        assert abs(diff.mean()) <= 5 * diff.std() / math.sqrt(n) + 1e-6 * np.abs(o_smp[:, c]).mean()
    hit_g, hit_o = np.isfinite(g_world[0]), np.isfinite(o_world[0])
    assert (hit_g == hit_o).mean() >= 0.995 and hit_o.mean() > 0.2
    both = hit_g & hit_o
    close = np.abs(g_world[:, both] - o_world[:, both]).max(0) <= 1e-3
    assert close.mean() >= 0.995
    fclose = np.abs(g_feat[:, both] - o_feat[:, both]).max(0) <= 2e-3
    assert fclose.mean() >= 0.99


def test_white_furnace_on_the_gpu():
    Wd, Hd = 64, 48
    sc = synth.vpt_scene(Wd, Hd, 0, seed=3, max_bounces=1 << 20)
    sc.update(albedo=1.0, color_lo=np.ones(3, np.float32), color_hi=np.ones(3, np.float32),
              light_rgb=np.zeros(3, np.float32), env_rgb=np.array([0.25, 0.5, 0.75], np.float32))
    smp, world, _ = _render_gpu(sc, Wd, Hd, 2)
    for c, e in enumerate((0.25, 0.5, 0.75)):
        assert np.all(smp[:, c] == np.float32(e))
    assert np.isfinite(world[0]).mean() > 0.2


def test_transmittance_of_a_homogeneous_box_on_the_gpu():
    eye = np.array([0.0, 0.0, 5.0], np.float32)
    ivp = np.linalg.inv(synth.perspective_view_proj(eye, (0.0, 0.0, 0.0), 0.01, 1.0)).astype(np.float32)
    blobs = np.zeros((16, 5), np.float32)
    blobs[0] = (0.0, 0.0, 0.0, 100.0, 2.0)
    mu = 0.8
    sc = {"seed": 7, "seed_hi": 11, "eye": eye, "inv_view_proj": ivp, "n_blobs": 1, "blobs": blobs, "mu_max": mu,
          "tf_lo": 0.0, "tf_hi": 0.5, "albedo": 0.0, "color_lo": np.ones(3, np.float32),
          "color_hi": np.ones(3, np.float32), "light_dir": np.array([1.0, 0.0, 0.0], np.float32),
          "light_rgb": np.zeros(3, np.float32), "env_rgb": np.ones(3, np.float32), "max_bounces": 1}
    smp, _, _ = _render_gpu(sc, 256, 256, 4)
    v = smp[:, 0].reshape(-1).astype(np.float64)
    T = math.exp(-2 * mu)
    assert set(np.unique(v)) <= {0.0, 1.0}
    assert abs(v.mean() - T) < 5 * math.sqrt(T * (1 - T) / v.size)


def test_full_hd_frame_and_pipeline_chain():
    """1920 x 1080 renders with finite outputs; and the chain render -> reconstruction ->
    velocity -> denoiser on 128 x 72 frames of a moving camera agrees with the same chain
    of oracles on >= 99 % of the pixels of every frame (paths that branch differently move
    a few pixels)."""
    sc = synth.vpt_scene(1920, 1080, 0, seed=4)
    smp = torch.empty(2, 5, 1080, 1920, device="cuda")
    world = torch.empty(3, 1080, 1920, device="cuda")
    W.wrls_render_vpt(sc, smp, world)
    torch.cuda.synchronize()
    assert torch.isfinite(smp).all() and 0.2 < torch.isfinite(world[0]).float().mean().item() < 1.0

    Wd, Hd, T = 128, 72, 8
    s = W.Stream(Wd, Hd)
    st = O.OracleStream(Wd, Hd, oracle_params_from(W.wrls_params_default()))
    rad = torch.empty(3, Hd, Wd, device="cuda")
    mot = torch.empty(2, Hd, Wd, device="cuda")
    out = torch.empty(3, Hd, Wd, device="cuda")
    g_smp = torch.empty(2, 5, Hd, Wd, device="cuda")
    g_world = torch.empty(3, Hd, Wd, device="cuda")
    for t in range(T):
        scene = synth.vpt_scene(Wd, Hd, t, seed=6, deg_per_frame=1.0)
        M_prev = synth.orbit_camera(t - 1, Wd, Hd, 1.0)
        W.wrls_render_vpt(scene, g_smp, g_world, frame=t)
        W.wrls_reconstruct(g_smp, rad)
        W.wrls_velocity_from_world(g_world, M_prev, mot)
        s.denoise(rad, mot, out)
        torch.cuda.synchronize()
        o_smp, o_world, _ = O.render_vpt(scene, Wd, Hd, 2, frame=t, features=False)
        o_rad, _ = O.reconstruct(o_smp, with_variance=False)
        o_mot = O.velocity(o_world, M_prev.astype(np.float32).astype(np.float64))
        ref, _, _ = st.frame(o_rad.astype(np.float32), o_mot.astype(np.float32))
        got = out.cpu().numpy()
        num = np.abs(got - ref).max(0)
        den = np.maximum(np.abs(ref).max(0), FLOOR)
        frac = float((num / den <= REL_TOL).mean())
        assert frac >= 0.99, (t, frac)
    s.close()
