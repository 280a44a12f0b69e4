"""Pins of the delta-tracking path tracer oracle (oracle/wrls_oracle_vpt.c), CPU only.

The renderer is a Monte Carlo estimator, so its pins are exact where the physics makes
every sample deterministic (a white furnace), and statistical (within 5 standard errors)
against closed forms elsewhere: the transmittance of a homogeneous box (Eq. 4's free-path
sampling) and single scattering in it (Eq. 3 with next-event estimation). The counter-based
generator is checked for uniformity, bit balance, avalanche and serial correlation."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2106_08034_gb300 import synth


def _narrow_camera(eye=(0.0, 0.0, 5.0), fov_deg=0.01):
    vp = synth.perspective_view_proj(eye, (0.0, 0.0, 0.0), fov_deg, 1.0)
    return np.asarray(eye, np.float32), np.linalg.inv(vp).astype(np.float32)


def _homogeneous_scene(mu, albedo, light=(0.0, 0.0, 0.0), env=(0.0, 0.0, 0.0), max_bounces=1,
                       light_dir=(1.0, 0.0, 0.0)):
    eye, ivp = _narrow_camera()
    blobs = np.zeros((16, 5), np.float32)
    blobs[0] = (0.0, 0.0, 0.0, 100.0, 2.0)      # density min(1, 2 exp(-|x|^2 / 2e4)) = 1 in the box
    return {"seed": 7, "seed_hi": 11, "eye": eye, "inv_view_proj": ivp, "n_blobs": 1, "blobs": blobs,
            "mu_max": float(mu), "tf_lo": 0.0, "tf_hi": 0.5, "albedo": float(albedo),
            "color_lo": np.ones(3, np.float32), "color_hi": np.ones(3, np.float32),
            "light_dir": np.asarray(light_dir, np.float32), "light_rgb": np.asarray(light, np.float32),
            "env_rgb": np.asarray(env, np.float32), "max_bounces": int(max_bounces)}


def test_philox_statistics():
    words = np.array([O.philox((i, 3, 5, 0), (0x1234, 0xABCD)) for i in range(1 << 14)], np.uint64).reshape(-1)
    # bit balance: every bit set in half of the words
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & 1).mean(0)
    sd = math.sqrt(0.25 / words.size)
    assert np.all(np.abs(bits - 0.5) < 5 * sd)
    # uniformity of the top byte (chi-square, 255 dof: mean 255, sd ~22.6)
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    exp = words.size / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert 255 - 5 * 22.6 < chi2 < 255 + 5 * 22.6
    # serial correlation of consecutive uniforms
    u = (words >> 8).astype(np.float64) / 2 ** 24
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / math.sqrt(u.size)
    # avalanche: one flipped counter bit changes about half of the 128 output bits
    flips = []
    for i in range(256):
        a = O.philox((i, 0, 0, 0), (1, 2))
        b = O.philox((i ^ (1 << (i % 32)), 0, 0, 0), (1, 2))
        flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64) < 2.5


def test_white_furnace_every_sample_is_the_environment():
    """No absorption (albedo 1, white), no light, uniform environment E: every path ends by
    leaving the volume with throughput 1, so every sample equals E exactly, whatever the
    heterogeneous density."""
    sc = synth.vpt_scene(48, 32, 0, seed=3, max_bounces=1 << 20)
    sc.update(albedo=1.0, color_lo=np.ones(3, np.float32), color_hi=np.ones(3, np.float32),
              light_rgb=np.zeros(3, np.float32), env_rgb=np.array([0.25, 0.5, 0.75], np.float32))
    smp, world, _ = O.render_vpt(sc, 48, 32, 2, features=False)
    for c, e in enumerate((0.25, 0.5, 0.75)):
        assert np.all(smp[:, c] == np.float32(e))
    assert np.isfinite(world[0]).mean() > 0.2          # the volume was hit


@pytest.mark.parametrize("mu", [0.3, 1.0, 2.0])
def test_transmittance_of_a_homogeneous_box(mu):
    """Absorbing box (albedo 0), environment E = 1, rays along -z through the centre (chord
    2): a sample is 1 when the ray crosses without a real collision, whose probability is
    exp(-2 mu) (Eq. 4's free-path sampling); else 0."""
    sc = _homogeneous_scene(mu, 0.0, env=(1.0, 1.0, 1.0))
    smp, _, _ = O.render_vpt(sc, 64, 64, 8, features=False)
    v = smp[:, 0].reshape(-1).astype(np.float64)
    assert set(np.unique(v)) <= {0.0, 1.0}
    T = math.exp(-2 * mu)
    assert abs(v.mean() - T) < 5 * math.sqrt(T * (1 - T) / v.size)


@pytest.mark.parametrize("mu,albedo", [(0.5, 0.8), (1.5, 0.6)])
def test_single_scattering_in_a_homogeneous_box(mu, albedo):
    """One real collision, then next-event estimation to a directional light along +x; rays
    along -z through the centre. The collision depth t on the chord [0, 2] has density
    mu exp(-mu t); the shadow ray from (0, 0, z) leaves after 1 (transmittance exp(-mu)):
      E[L] = albedo E_L / (4 pi) exp(-mu) (1 - exp(-2 mu))."""
    EL = 4.0 * math.pi
    sc = _homogeneous_scene(mu, albedo, light=(EL, EL, EL))
    smp, _, _ = O.render_vpt(sc, 64, 64, 8, features=False)
    v = smp[:, 1].reshape(-1).astype(np.float64)
    ref = albedo * EL / (4 * math.pi) * math.exp(-mu) * (1 - math.exp(-2 * mu))
    assert abs(v.mean() - ref) < 5 * v.std() / math.sqrt(v.size) + 1e-12


def test_first_collision_outputs_are_consistent():
    """World positions lie inside the volume where the opacity is positive (a real collision
    needs mu_t > 0); the depth feature is their distance from the eye; normals are unit
    vectors; pixels without a collision have NaN positions and zero features; a fixed seed
    and frame reproduce the frame exactly, another frame does not."""
    W, H = 40, 30
    sc = synth.vpt_scene(W, H, 0, seed=5)
    smp, world, feat = O.render_vpt(sc, W, H, 2)
    hit = np.isfinite(world[0])
    assert 0.2 < hit.mean() < 1.0
    P = world[:, hit].astype(np.float64)
    assert np.all(np.abs(P) <= 1.0 + 1e-6)
    eye = np.asarray(sc["eye"], np.float64)[:, None]
    assert np.allclose(feat[0, hit], np.linalg.norm(P - eye, axis=0), rtol=1e-5)
    nrm = np.linalg.norm(feat[1:4, hit], axis=0)
    assert np.all((np.abs(nrm - 1) < 1e-5) | (nrm == 0))
    assert np.all(feat[:, ~hit] == 0) and np.all(np.isnan(world[:, ~hit]))
    b = sc["blobs"][:sc["n_blobs"]].astype(np.float64)
    d2 = ((P.T[:, None, :] - b[None, :, :3]) ** 2).sum(-1)
    rho = np.minimum(1.0, (b[None, :, 4] * np.exp(-d2 / (2 * b[None, :, 3] ** 2))).sum(-1))
    assert np.all(rho > sc["tf_lo"])
    smp2, _, _ = O.render_vpt(sc, W, H, 2)
    smp3, _, _ = O.render_vpt(sc, W, H, 2, frame=1)
    assert np.array_equal(smp, smp2) and not np.array_equal(smp, smp3)
