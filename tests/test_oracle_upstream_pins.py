"""Pins of the oracle of the denoiser's input steps (oracle/wrls_oracle_upstream.c): the pixel
reconstruction filter and the velocity from first-collision world positions (CPU only).

Checks against scipy's correlation with the separable Gaussian kernel, exact constants,
numpy's sample variance, and projections whose result is known analytically. Test
geometry is built here with numpy, independently of the generator's camera code."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle as O


def _samples(rng, spp, H, W, zero_offsets=False):
    s = np.empty((spp, 5, H, W), np.float32)
    s[:, :3] = rng.uniform(0.0, 2.0, (spp, 3, H, W))
    s[:, 3:] = 0.0 if zero_offsets else rng.uniform(-0.5, 0.5, (spp, 2, H, W))
    return s


@pytest.mark.parametrize("sigma", [0.5, 0.8])
def test_reconstruction_at_pixel_centres_is_a_normalised_separable_gaussian(sigma):
    """One sample per pixel at its centre: I~ = correlate(f, g g^T) / correlate(1, g g^T)
    with g = [exp(-1/(2 sigma^2)), 1, exp(-1/(2 sigma^2))] and zero outside the image."""
    rng = np.random.default_rng(1)
    H, W = 9, 13
    smp = _samples(rng, 1, H, W, zero_offsets=True)
    out, _ = O.reconstruct(smp, sigma=sigma)
    g = np.array([math.exp(-1 / (2 * sigma ** 2)), 1.0, math.exp(-1 / (2 * sigma ** 2))])
    K = np.outer(g, g)
    norm = ndi.correlate(np.ones((H, W)), K, mode="constant", cval=0.0)
    for c in range(3):
        ref = ndi.correlate(smp[0, c].astype(np.float64), K, mode="constant", cval=0.0) / norm
        assert np.allclose(out[c], ref, rtol=1e-13, atol=1e-13)


def test_reconstruction_reproduces_a_constant_and_respects_the_support():
    rng = np.random.default_rng(2)
    H, W, spp = 7, 10, 3
    smp = _samples(rng, spp, H, W)
    smp[:, 0], smp[:, 1], smp[:, 2] = 0.25, 1.5, 3.0
    out, _ = O.reconstruct(smp)
    assert np.allclose(out[0], 0.25, atol=1e-14) and np.allclose(out[2], 3.0, atol=1e-14)
    # support radius 0.6 with samples at the centres: only the pixel's own samples count,
    # whatever sigma; a very narrow sigma with radius 1.5 gives the same to double precision
    smp = _samples(rng, spp, H, W, zero_offsets=True)
    own = smp[:, :3].astype(np.float64).mean(0)
    out_r, _ = O.reconstruct(smp, sigma=2.0, radius=0.6)
    out_s, _ = O.reconstruct(smp, sigma=0.05, radius=1.5)
    assert np.allclose(out_r, own, rtol=1e-14, atol=1e-14)
    assert np.allclose(out_s, own, rtol=1e-12, atol=1e-12)


def test_reconstruction_variance_and_missing_samples():
    """variance = unbiased sample variance of the pixel's own finite samples, averaged over
    the channels, divided by their count (numpy var, ddof=1); NaN with < 2 finite samples;
    a window without any finite sample gives a non-finite estimate."""
    rng = np.random.default_rng(3)
    H, W, spp = 5, 6, 4
    smp = _samples(rng, spp, H, W)
    _, var = O.reconstruct(smp)
    ref = smp[:, :3].astype(np.float64).var(axis=0, ddof=1).mean(0) / spp
    assert np.allclose(var, ref, rtol=1e-12, atol=0)
    smp[0, 1, 2, 3] = np.nan                      # one sample of pixel (3, 2) missing
    _, var = O.reconstruct(smp)
    keep = smp[1:, :3, 2, 3].astype(np.float64)
    assert abs(var[2, 3] - keep.var(axis=0, ddof=1).mean() / 3) < 1e-12
    smp[1:, 0, 2, 3] = np.inf                     # a single finite sample left
    out, var = O.reconstruct(smp)
    assert np.isnan(var[2, 3]) and np.all(np.isfinite(out))
    smp = _samples(rng, 1, 4, 4)
    smp[:, 0] = np.nan                            # nothing finite anywhere
    out, _ = O.reconstruct(smp)
    assert not np.any(np.isfinite(out))


def _pixel_ndc(W, H):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    return (xs + 0.5) / W * 2 - 1, 1 - (ys + 0.5) / H * 2, xs, ys


def test_velocity_identity_projection_and_ndc_shift():
    """M = I: a world point at the NDC position of pixel j's centre shifted by (sx, sy) in NDC
    lands (sx W / 2, -sy H / 2) pixels away (row 0 at the top)."""
    W, H = 16, 10
    nx, ny, _, _ = _pixel_ndc(W, H)
    sx, sy = 0.125, -0.25
    world = np.stack([nx + sx, ny + sy, np.zeros_like(nx)]).astype(np.float32)
    mot = O.velocity(world, np.eye(4))
    # world was rounded to binary32; the expected shift follows from the rounded coordinates
    wx = world[0].astype(np.float64)
    wy = world[1].astype(np.float64)
    exp_x = (wx + 1) * W / 2 - 0.5 - np.arange(W)[None, :]
    exp_y = (1 - wy) * H / 2 - 0.5 - np.arange(H)[:, None]
    assert np.allclose(mot[0], exp_x, atol=1e-12) and np.allclose(mot[1], exp_y, atol=1e-12)
    assert np.allclose(mot[0], sx * W / 2, atol=1e-5) and np.allclose(mot[1], -sy * H / 2, atol=1e-5)


def test_velocity_perspective_divide_static_camera_and_misses():
    """Static camera: points on the rays through the pixel centres (unprojected here with
    numpy's inverse of M) have zero motion; a point behind the camera (w <= 0) gives NaN; a
    pixel without a collision gives 0 or NaN by the miss policy."""
    W, H = 12, 8
    f, aspect, near, far = 1.0 / math.tan(math.radians(25)), W / H, 0.1, 50.0
    P = np.array([[f / aspect, 0, 0, 0], [0, f, 0, 0],
                  [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)], [0, 0, -1, 0]])
    th = math.radians(20)
    V = np.array([[math.cos(th), 0, -math.sin(th), 0.3], [0, 1, 0, -0.2],
                  [math.sin(th), 0, math.cos(th), -5.0], [0, 0, 0, 1]])
    M = P @ V
    nx, ny, _, _ = _pixel_ndc(W, H)
    rng = np.random.default_rng(4)
    nz = rng.uniform(0.8, 0.99, (H, W))
    clip = np.stack([nx, ny, nz, np.ones_like(nz)]).reshape(4, -1)
    Xh = np.linalg.inv(M) @ clip
    world = (Xh[:3] / Xh[3]).reshape(3, H, W).astype(np.float32)
    mot = O.velocity(world, M)
    assert np.abs(mot).max() < 2e-4          # binary32 world positions
    behind = world.copy()
    cam = -np.linalg.inv(V[:3, :3]) @ V[:3, 3]                 # camera centre
    fwd = -np.linalg.inv(V[:3, :3])[:, 2]                      # viewing direction
    behind[:, 0, 0] = (cam - 2.0 * fwd).astype(np.float32)
    behind[:, 1, 1] = np.nan
    m0 = O.velocity(behind, M, miss_policy=0)
    m1 = O.velocity(behind, M, miss_policy=1)
    assert np.all(np.isnan(m0[:, 0, 0])) and np.all(m0[:, 1, 1] == 0.0) and np.all(np.isnan(m1[:, 1, 1]))


def test_velocity_of_a_screen_parallel_camera_shift():
    """Orthographic camera (clip = S (X - c)) that was at c = (d, 0, 0) in the previous frame
    and is at the origin now: every point sat d S_x W / 2 pixels further left in the previous
    image, so the backward motion is v_x = -d S_x W / 2, v_y = 0."""
    W, H = 20, 10
    S = np.diag([0.2, 0.4, 0.1, 1.0])
    d = 1.5
    T_prev = np.eye(4)
    T_prev[0, 3] = -d                       # previous camera at x = +d: clip_x = S_x (X - d)
    M_prev = S @ T_prev
    nx, ny, _, _ = _pixel_ndc(W, H)
    # current camera at the origin: world point of pixel j has X = ndc_x / S_x
    world = np.stack([nx / 0.2, ny / 0.4, np.full_like(nx, 3.0)]).astype(np.float32)
    mot = O.velocity(world, M_prev)
    assert np.allclose(mot[0], -d * 0.2 * W / 2, atol=1e-4) and np.allclose(mot[1], 0.0, atol=1e-4)


def test_reconstruction_single_offset_sample_closed_form():
    """All samples at their pixel centres with colour 0, except pixel p's sample: colour F at
    offset (ox, oy). At the pixel j = p + (1, 0) (interior) the sample sits at
    (ox - 1, oy) from j's centre, so
        I~_j = g(ox - 1) g(oy) F / (g(ox - 1) g(oy) + (1 + 2 g(1))^2 - g(1) g(0)),
    g(d) = exp(-d^2 / (2 sigma^2)): the centre-weight sum of the 3x3 window with p's centre
    term replaced by its actual one."""
    H, W, sigma = 7, 9, 0.5
    smp = np.zeros((1, 5, H, W), np.float32)
    py, px, ox, oy, F = 3, 4, 0.375, -0.25, 2.0
    smp[0, 0, py, px] = F
    smp[0, 3, py, px], smp[0, 4, py, px] = ox, oy
    out, _ = O.reconstruct(smp, sigma=sigma)

    def g(d):
        return math.exp(-d * d / (2 * sigma * sigma))
    w = g(ox - 1) * g(oy)
    ref = w * F / (w + (1 + 2 * g(1)) ** 2 - g(1) * g(0))
    assert abs(out[0, py, px + 1] - ref) < 1e-14
    # and at j = p - (1, 0) the same sample sits at (ox + 1, oy)
    w2 = g(ox + 1) * g(oy)
    ref2 = w2 * F / (w2 + (1 + 2 * g(1)) ** 2 - g(1) * g(0))
    assert abs(out[0, py, px - 1] - ref2) < 1e-14


def test_reconstruction_skips_samples_with_nonfinite_offsets():
    """A sample whose offset is not finite is missing like one with a non-finite colour:
    the estimate equals the one where that sample's colour is NaN instead."""
    rng = np.random.default_rng(6)
    smp = _samples(rng, 3, 6, 7)
    a, b = smp.copy(), smp.copy()
    a[1, 3, 2, 4] = np.nan
    b[1, 0, 2, 4] = np.nan
    oa, va = O.reconstruct(a)
    ob, vb = O.reconstruct(b)
    assert np.array_equal(oa, ob) and np.array_equal(va, vb) and np.all(np.isfinite(oa))
