"""Pins of the FP64 oracle to what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form of the
recursion (Sherman-Morrison / weighted least squares), a brute-force least-squares solve
of the stacked design matrix of Eq. 7, scipy filters, exact equivariances, or special
values of Eq. 12-14. Sizes are small so the whole file runs in seconds.
"""
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle as O
from paper_2106_08034_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frames(spec):
    sc = synth.Scene(spec)
    return [sc.frame(t) for t in range(spec.frames)]


def _run(frames, W, H, prm, hook=None):
    st = O.OracleStream(W, H, prm)
    hist = []
    for t, f in enumerate(frames):
        rad = f["radiance"].numpy()
        mot = f["motion"].numpy()
        if hook is not None:
            rad, mot = hook(t, rad.copy(), mot.copy())
        out, w, valid = st.frame(rad, mot)
        hist.append(dict(out=out, w=w, valid=valid, beta=st.beta.copy(), P=st.P.copy(),
                         z=st.z.copy(), rad=rad, mot=mot))
    return hist


def _p_vectors(z):                      # Sec. 5.1: p = [1, z]
    return np.concatenate([np.ones((z.shape[0], 1)), z], 1)


# --- constants the paper prints ------------------------------------------------------

def test_paper_constants_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                vals[name] = float(value)
    prm = O.OracleParams()
    assert prm.lambda_ == vals["lambda"]
    assert prm.h == vals["h"]
    assert prm.alpha == vals["alpha"]
    assert 2 * prm.radius + 1 == vals["blend_window"]
    st = O.OracleStream(2, 2)
    assert st.beta.shape[-1] == vals["predictor_dim"] and st.P.shape[-1] == vals["predictor_dim"]


# --- Eq. 8-11, 14 against their batch closed form -------------------------------------

@pytest.mark.parametrize("frames,init_mode", [(8, 0), (120, 0), (8, 1)])
def test_recursion_equals_batch_weighted_least_squares(frames, init_mode):
    """Static camera, no resets after frame 0: by the matrix inversion lemma,
    P(t)^-1 = lambda^(t+1) P0^-1 + sum_s lambda^(t-s) w_s p_s p_s^T and
    beta_c(t) = P(t) (lambda^(t+1) P0^-1 beta0_c + sum_s lambda^(t-s) w_s p_s I~_c,s).
    Uses the z_s and w_s the recursion produced; checks Eq. 8, 9, 11 and 14."""
    W = H = 8
    spec = synth.SceneSpec(W, H, frames, seed=11, motion="static", firefly_frac=0.1)
    prm = O.OracleParams(init_mode=init_mode)
    hist = _run(_frames(spec), W, H, prm)
    lam, delta = prm.lambda_, prm.p0_delta
    n = W * H
    beta0 = np.zeros((n, 3, 4))
    if init_mode == 1:
        for c in range(3):
            beta0[:, c, c + 1] = 1.0
    A = np.zeros((n, 4, 4))
    b = np.zeros((n, 3, 4))
    for t, h in enumerate(hist):
        p = _p_vectors(h["z"])                          # p_t = [1, z_t] (z after frame t)
        w = h["w"].reshape(n)
        I = h["rad"].reshape(3, n).T.astype(np.float64)
        A = lam * A + w[:, None, None] * p[:, :, None] * p[:, None, :]
        b = lam * b + w[:, None, None] * I[:, :, None] * p[:, None, :]
        prior = lam ** (t + 1) / delta
        At = A + prior * np.eye(4)[None]
        bt = b + prior * beta0
        beta_ls = np.linalg.solve(At, bt.transpose(0, 2, 1)).transpose(0, 2, 1)
        P_ls = np.linalg.inv(At)
        scale_b = np.maximum(1.0, np.abs(beta_ls).max())
        assert np.abs(h["beta"] - beta_ls).max() / scale_b < 1e-9, t
        assert np.abs(h["P"] - P_ls).max() / np.abs(P_ls).max() < 1e-9, t


def test_recursion_equals_bruteforce_stacked_lstsq():
    """Eq. 7: stack the weighted predictor rows sqrt(lambda^(t-s) w_s) p_s over time plus
    the prior rows, and solve by QR least squares; beta(t) must agree."""
    W, H, T = 8, 8, 12
    spec = synth.SceneSpec(W, H, T, seed=12, motion="static", firefly_frac=0.05)
    prm = O.OracleParams()
    hist = _run(_frames(spec), W, H, prm)
    lam, delta = prm.lambda_, prm.p0_delta
    t = T - 1
    for j in range(0, W * H, 7):
        rows, tgt = [], []
        for s in range(t + 1):
            ws = hist[s]["w"].reshape(-1)[j] * lam ** (t - s)
            ps = np.concatenate([[1.0], hist[s]["z"][j]])
            rows.append(math.sqrt(ws) * ps)
            tgt.append(math.sqrt(ws) * hist[s]["rad"].reshape(3, -1)[:, j].astype(np.float64))
        sp = math.sqrt(lam ** (t + 1) / delta)
        X = np.vstack(rows + [sp * np.eye(4)])
        Y = np.vstack(tgt + [np.zeros((4, 3))])          # prior beta0 = 0
        beta_ls, *_ = np.linalg.lstsq(X, Y, rcond=None)  # (4, 3)
        assert np.allclose(hist[t]["beta"][j], beta_ls.T, rtol=1e-9, atol=1e-9), j


@pytest.mark.parametrize("init_mode", [0, 1])
def test_intercept_only_is_weighted_running_mean(init_mode):
    """p = [1] (no feature): beta(t) is the lambda- and w-weighted mean of the samples with
    the prior, a scalar geometric sum."""
    W, H, T = 6, 5, 30
    spec = synth.SceneSpec(W, H, T, seed=13, motion="static", firefly_frac=0.1)
    prm = O.OracleParams(feature_mode=1, init_mode=init_mode)
    hist = _run(_frames(spec), W, H, prm)
    lam, delta = prm.lambda_, prm.p0_delta
    n = W * H
    beta0 = np.zeros((n, 3)) if init_mode == 0 else hist[0]["rad"].reshape(3, n).T.astype(np.float64)
    num = np.zeros((n, 3))
    den = np.zeros(n)
    for t, h in enumerate(hist):
        w = h["w"].reshape(n)
        I = h["rad"].reshape(3, n).T.astype(np.float64)
        num = lam * num + w[:, None] * I
        den = lam * den + w
        pr = lam ** (t + 1) / delta
        ref = (num + pr * beta0) / (den + pr)[:, None]
        assert np.abs(h["beta"][:, :, 0] - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())
        assert np.allclose(h["P"][:, 0, 0], 1.0 / (den + pr), rtol=1e-11)


# --- Eq. 12 ---------------------------------------------------------------------------

def _uniform_frames(W, H, values):
    out = []
    for v in values:
        rad = np.empty((3, H, W), np.float32)
        rad[:] = np.asarray(v, np.float32)[:, None, None]
        out.append(dict(radiance=_T(rad), motion=_T(np.zeros((2, H, W), np.float32))))
    return out


class _T:
    """Minimal tensor stand-in with .numpy() for hand-made frames."""
    def __init__(self, a):
        self.a = a

    def numpy(self):
        return self.a


def test_feature_geometric_decay_without_clamp():
    """Eq. 12 with Psi off and a step from A to B: z(T0+k) = B + alpha^(k+1) (A - B)."""
    W, H, T0 = 4, 3, 3
    A, B = np.array([0.2, 0.5, 0.7]), np.array([0.9, 0.1, 0.4])
    prm = O.OracleParams(clamp_mode=1)
    hist = _run(_uniform_frames(W, H, [A] * T0 + [B] * 6), W, H, prm)
    A32, B32 = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    for k in range(6):
        ref = B32 + prm.alpha ** (k + 1) * (A32 - B32)
        assert np.abs(hist[T0 + k]["z"] - ref[None]).max() < 1e-14


def test_feature_clamp_is_projection_on_neighbourhood_box():
    """Psi clamps the history to the per-channel min/max of I~ over the 3x3 neighbours
    inside the image; clamping is the projection median(lo, z, hi). lo/hi come from
    scipy's min/max filters (edge replication leaves the window's extrema unchanged)."""
    W, H = 16, 12
    spec = synth.SceneSpec(W, H, 5, seed=14, motion="static")
    prm = O.OracleParams()
    hist = _run(_frames(spec), W, H, prm)
    for t in range(1, 5):
        rad = hist[t]["rad"].astype(np.float64)
        lo = np.stack([ndi.minimum_filter(rad[c], size=3, mode="nearest") for c in range(3)])
        hi = np.stack([ndi.maximum_filter(rad[c], size=3, mode="nearest") for c in range(3)])
        zq = hist[t - 1]["z"].reshape(H, W, 3).transpose(2, 0, 1)
        ref = prm.alpha * np.median(np.stack([lo, zq, hi]), axis=0) + (1 - prm.alpha) * rad
        got = hist[t]["z"].reshape(H, W, 3).transpose(2, 0, 1)
        assert np.abs(got - ref).max() < 1e-14


# --- Eq. 13 ---------------------------------------------------------------------------

def test_weight_special_values():
    W, H = 5, 4
    prm = O.OracleParams(clamp_mode=1)
    a = 0.2
    r3 = math.sqrt(3.0)
    # choose b so that d = ||I~ - z|| / (min(||I~||, ||z||) + eps) = h exactly (z < I~)
    al, h, eps = prm.alpha, prm.h, prm.eps
    b = (h * eps + al * a * r3 * (1 + h)) / (r3 * (al - h * (1 - al)))
    hist = _run(_uniform_frames(W, H, [[a] * 3, [b] * 3]), W, H, prm)
    assert np.all(hist[0]["w"] == 1.0)          # frame 0: z = I~, d = 0
    a32, b32 = float(np.float32(a)), float(np.float32(b))
    z1 = al * a32 + (1 - al) * b32
    d = al * (b32 - a32) * r3 / (z1 * r3 + eps)
    assert abs(hist[1]["w"][0, 0] - math.exp(-d * d / (h * h))) < 1e-15
    assert abs(d - h) < 1e-6                     # the construction hits d = h: w ~ 1/e
    assert abs(hist[1]["w"][0, 0] - math.exp(-1.0)) < 1e-5
    # RLS mode: w == 1 whatever the distance
    hist_rls = _run(_uniform_frames(W, H, [[a] * 3, [b] * 3]), W, H, O.OracleParams(weight_mode=1))
    assert np.all(hist_rls[1]["w"] == 1.0)


def test_missing_sample_has_zero_weight_and_freezes_beta():
    W, H = 10, 8
    spec = synth.SceneSpec(W, H, 5, seed=15, motion="static")
    prm = O.OracleParams()

    def hook(t, rad, mot):
        if t == 3:
            rad[0, 4, 5] = np.nan
        return rad, mot
    hist = _run(_frames(spec), W, H, prm, hook)
    j = 4 * W + 5
    assert hist[3]["w"][4, 5] == 0.0
    assert np.array_equal(hist[3]["beta"][j], hist[2]["beta"][j])
    assert np.allclose(hist[3]["P"][j], hist[2]["P"][j] / prm.lambda_, rtol=1e-15, atol=0)
    assert np.all(np.isfinite(hist[3]["out"]))
    assert np.all(np.isfinite(hist[4]["out"]))


# --- reprojection --------------------------------------------------------------------

def test_translation_equivariance_integer_pan():
    """Frames B_t(x, y) = A_t(x + t, y + t) with v = (+1, +1) (previous position j + v)
    must give out_B(x, y, t) = out_A(x + t, y + t, t) where no window met a border.
    Pins the reprojection direction, the axes and that models (not colours) move."""
    T, W, H = 6, 20, 16
    WA, HA = W + T + 8, H + T + 8
    specA = synth.SceneSpec(WA, HA, T, seed=16, motion="static", firefly_frac=0.05)
    fa = _frames(specA)
    prm = O.OracleParams()
    histA = _run(fa, WA, HA, prm)
    fb = []
    for t in range(T):
        rad = fa[t]["radiance"].numpy()[:, t:t + H, t:t + W].copy()
        mot = np.ones((2, H, W), np.float32) if t > 0 else np.zeros((2, H, W), np.float32)
        fb.append(dict(radiance=_T(rad), motion=_T(mot)))
    histB = _run(fb, W, H, prm)
    for t in range(T):
        m = 3
        ys, xs = slice(m, H - m - 1 - t), slice(m, W - m - 1 - t)
        got = histB[t]["out"][:, ys, xs]
        ref = histA[t]["out"][:, t + m:t + H - m - 1 - t, t + m:t + W - m - 1 - t]
        assert got.size > 0
        assert np.abs(got - ref).max() < 1e-13, t
        assert np.all(histB[t]["valid"][ys, xs] == (t > 0))


def test_rotation_equivariance_non_square():
    """Rotating every input by 90 degrees (motion v -> (v_y, -v_x)) rotates the output.
    Motions are multiples of 1/4 so binary32 addresses are exact in both frames."""
    T, W, H = 5, 14, 10
    spec = synth.SceneSpec(W, H, T, seed=17, motion="static", firefly_frac=0.05)
    fr = _frames(spec)
    rng = np.random.default_rng(0)
    frames_a, frames_b = [], []
    for t in range(T):
        rad = fr[t]["radiance"].numpy()
        mot = (rng.integers(-6, 7, size=(2, H, W)) / 4.0).astype(np.float32)
        frames_a.append(dict(radiance=_T(rad), motion=_T(mot)))
        rad_r = np.ascontiguousarray(np.rot90(rad, axes=(1, 2)))
        mot_r = np.ascontiguousarray(np.stack([np.rot90(mot[1]), -np.rot90(mot[0])]))
        frames_b.append(dict(radiance=_T(rad_r), motion=_T(mot_r)))
    prm = O.OracleParams()
    ha = _run(frames_a, W, H, prm)
    hb = _run(frames_b, H, W, prm)
    for t in range(T):
        ref = np.rot90(ha[t]["out"], axes=(1, 2))
        assert np.abs(hb[t]["out"] - ref).max() < 1e-12, t
        assert np.array_equal(hb[t]["valid"], np.rot90(ha[t]["valid"]))


def test_invalid_reprojection_restarts_pixel():
    """A pixel whose q = j + v leaves the image restarts: its state equals the state a
    fresh stream computes for the same frame."""
    W, H = 12, 9
    spec = synth.SceneSpec(W, H, 4, seed=18, motion="static")
    fr = _frames(spec)
    prm = O.OracleParams()

    def hook(t, rad, mot):
        if t == 3:
            mot[0, :, :3] = -5.0          # q_x < 0 for the 3 leftmost columns
            mot[1, 0, 6] = -0.5           # q_y < 0
        return rad, mot
    hist = _run(fr, W, H, prm, hook)
    fresh = O.OracleStream(W, H, prm)
    fresh.frame(hist[3]["rad"], hist[3]["mot"])
    inval = ~hist[3]["valid"]
    assert inval[:, :3].all() and inval[0, 6] and inval.sum() == 3 * H + 1
    idx = np.flatnonzero(inval.reshape(-1))
    assert np.array_equal(hist[3]["beta"][idx], fresh.beta[idx])
    assert np.array_equal(hist[3]["P"][idx], fresh.P[idx])
    assert np.array_equal(hist[3]["z"][idx], fresh.z[idx])


# --- blend (Sec. 5.3) -------------------------------------------------------------------

def _gauss_kernel(sigma, r):
    g1 = np.exp(-np.arange(-r, r + 1) ** 2 / (2 * sigma * sigma))
    return np.outer(g1, g1)                 # separable


def test_blend_spatial_weights_match_normalised_convolution():
    """Uniform z (range weight 1): the blend is a normalised 5x5 Gaussian convolution of
    the predictions p . beta_k, with out-of-image taps dropped."""
    W, H = 11, 9
    rng = np.random.default_rng(1)
    beta = rng.normal(size=(W * H, 3, 4))
    zc = np.array([0.3, 0.6, 0.2])
    z = np.tile(zc, (W * H, 1))
    prm = O.OracleParams()
    out = O.blend(prm, beta, z, W, H)
    p = np.concatenate([[1.0], zc])
    K = _gauss_kernel(prm.sigma_s, prm.radius)
    den = ndi.correlate(np.ones((H, W)), K, mode="constant", cval=0.0)
    for c in range(3):
        pred = (beta[:, c, :] @ p).reshape(H, W)
        ref = ndi.correlate(pred, K, mode="constant", cval=0.0) / den
        assert np.abs(out[c] - ref).max() < 1e-12


def test_blend_range_weight_across_an_edge():
    """Two regions whose features are at Eq. 13 distance d = h_s get range weight e^-1;
    each pixel's neighbours predict with that pixel's own p (cross-prediction)."""
    W, H = 12, 8
    prm = O.OracleParams()
    r3 = math.sqrt(3.0)
    a = 0.3
    b = a * (1.0 + prm.h_s) + prm.h_s * prm.eps / r3      # |b-a| r3 / (a r3 + eps) = h_s
    mA = np.zeros((H, W), bool)
    mA[:, :5] = True
    z = np.where(mA.reshape(-1, 1), a, b) * np.ones((1, 3))
    rng = np.random.default_rng(2)
    beta = rng.normal(size=(W * H, 3, 4))
    out = O.blend(prm, beta, z, W, H)
    d = abs(b - a) * r3 / (a * r3 + prm.eps)
    e = math.exp(-d * d / prm.h_s ** 2)
    assert abs(e - math.exp(-1.0)) < 1e-12
    K = _gauss_kernel(prm.sigma_s, prm.radius)
    fA, fB = mA.astype(float), (~mA).astype(float)
    for region, zv, same, other in [(mA, a, fA, fB), (~mA, b, fB, fA)]:
        p = np.array([1.0, zv, zv, zv])
        den = ndi.correlate(same, K, mode="constant") + e * ndi.correlate(other, K, mode="constant")
        for c in range(3):
            pred = (beta[:, c, :] @ p).reshape(H, W)
            num = (ndi.correlate(pred * same, K, mode="constant") +
                   e * ndi.correlate(pred * other, K, mode="constant"))
            assert np.abs(out[c][region] - (num / den)[region]).max() < 1e-12


def test_zero_noise_returns_clean_input():
    """Feature pass-through start (prediction = z) and I~ = I on a static camera: z stays
    I, every residual is 0, so out = I exactly for the 5x5 cross-prediction blend and for
    the temporal-only output; blending own predictions (p_k beta_k) is not the identity."""
    W, H, T = 24, 18, 6
    spec = synth.SceneSpec(W, H, T, seed=19, motion="static", noiseless=True)
    fr = _frames(spec)
    for radius in (2, 0):
        hist = _run(fr, W, H, O.OracleParams(init_mode=1, radius=radius))
        for t in range(T):
            truth = fr[t]["truth"].numpy().astype(np.float64)
            assert np.abs(hist[t]["out"] - truth).max() < 1e-12
    hist = _run(fr, W, H, O.OracleParams(init_mode=1, blend_mode=1))
    assert np.abs(hist[-1]["out"] - fr[-1]["truth"].numpy()).max() > 1e-3


def test_zero_noise_temporal_output_closed_form_from_zero_start():
    """Zero model start, I~ = I constant in time, temporal-only output (radius 0): p is an
    eigenvector of P(t)^-1 = lambda^(t+1)/delta I + S_t p p^T, S_t = sum_s lambda^(t-s), so
    p . beta(t) = I S_t |p|^2 / (lambda^(t+1)/delta + S_t |p|^2)."""
    W, H, T = 16, 12, 40
    spec = synth.SceneSpec(W, H, T, seed=20, motion="static", noiseless=True)
    fr = _frames(spec)
    prm = O.OracleParams(radius=0)
    hist = _run(fr, W, H, prm)
    lam, delta = prm.lambda_, prm.p0_delta
    I = fr[0]["truth"].numpy().astype(np.float64)
    p2 = 1.0 + (I * I).sum(0)
    for t, h in enumerate(hist):
        S = (1 - lam ** (t + 1)) / (1 - lam)
        ref = I * (S * p2 / (lam ** (t + 1) / delta + S * p2))[None]
        assert np.abs(h["out"] - ref).max() < 1e-12, t


# --- invariants ----------------------------------------------------------------------

def test_invariants_on_a_moving_noisy_sequence():
    W, H, T = 40, 30, 16
    spec = synth.SceneSpec(W, H, T, seed=21, motion="orbit", firefly_frac=0.05)
    hist = _run(_frames(spec), W, H, O.OracleParams())
    lam = O.OracleParams().lambda_
    for h in hist:
        P = h["P"]
        assert np.abs(P - P.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(P).max()
        ev = np.linalg.eigvalsh(0.5 * (P + P.transpose(0, 2, 1)))
        assert ev.min() > 0
        assert np.all((h["w"] >= 0) & (h["w"] <= 1))
        z = h["z"]
        p = _p_vectors(z)
        s = np.einsum("na,nab,nb->n", p, P, p)
        assert np.all(lam + h["w"].reshape(-1) * s >= lam)
        assert np.all(np.isfinite(h["out"]))
    assert not hist[-1]["valid"].all() and hist[-1]["valid"].any()


def test_paper_qualitative_claims():
    """Sec. 5.3 / Fig. 9: wRLS beats RLS on spike noise; the 5x5 blend lowers the error of
    the temporal-only output; the output beats the input (Sec. 7.4)."""
    W, H, T = 48, 40, 16
    spec = synth.SceneSpec(W, H, T, seed=22, motion="pan", firefly_frac=0.05)
    fr = _frames(spec)

    def relmse(prm):
        hist = _run(fr, W, H, prm)
        return np.mean([np.mean((h["out"] - fr[t]["truth"].numpy()) ** 2 /
                                (fr[t]["truth"].numpy() ** 2 + 1e-2)) for t, h in enumerate(hist)][-6:])
    inp = np.mean([np.mean((f["radiance"].numpy() - f["truth"].numpy()) ** 2 /
                           (f["truth"].numpy() ** 2 + 1e-2)) for f in fr][-6:])
    wrls = relmse(O.OracleParams())
    rls = relmse(O.OracleParams(weight_mode=1))
    temporal = relmse(O.OracleParams(radius=0))
    assert wrls < 0.5 * rls
    assert wrls < temporal
    assert wrls < 0.2 * inp


def test_channel_permutation_equivariance():
    """R2 (one P shared by the three channel models): permuting the colour channels of every
    input permutes the output channels, because the weight depends on colour norms only and
    the shared P of p = [1, z] is only reordered. A channel index mix-up or a P that is not
    shared consistently breaks this."""
    W, H, T = 10, 8, 12
    spec = synth.SceneSpec(W, H, T, seed=31, motion="orbit", firefly_frac=0.1)
    fr = _frames(spec)
    perm = [2, 0, 1]
    a = O.OracleStream(W, H)
    b = O.OracleStream(W, H)
    for f in fr:
        rad, mot = f["radiance"].numpy(), f["motion"].numpy()
        oa, wa, _ = a.frame(rad, mot)
        ob, wb, _ = b.frame(np.ascontiguousarray(rad[perm]), mot)
        assert np.allclose(wb, wa, rtol=1e-12, atol=1e-14)
        assert np.allclose(ob, oa[perm], rtol=1e-9, atol=1e-12)
