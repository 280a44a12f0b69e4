"""Pins of the extended FP64 oracle (oracle/wrls_oracle_ext.c): G-buffer predictor entries
p = [1, z, g] up to d = 8, the sample-variance weight and nearest-pixel reprojection
(CPU only).

Each test checks the oracle against something other than itself: the paper-predictor
oracle where the extension reduces to it, the weighted-least-squares closed form and a QR
solve of the stacked design matrix of Eq. 7 at d = 8, special values of the variance
weight, the pixel that nearest-pixel reprojection must pick, and blends whose result is
known exactly.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2106_08034_gb300 import synth


def _frames(spec):
    sc = synth.Scene(spec)
    return [sc.frame(t) for t in range(spec.frames)]


def _run_ext(frames, W, H, prm, hook=None):
    st = O.OracleExtStream(W, H, prm)
    hist = []
    for t, f in enumerate(frames):
        rad, mot = f["radiance"].numpy().copy(), f["motion"].numpy().copy()
        var, g = f["variance"].numpy().copy(), f["features"].numpy().copy()
        if hook is not None:
            rad, mot, var, g = hook(t, rad, mot, var, g)
        out, w, valid = st.frame(rad, mot, var, g)
        hist.append(dict(out=out, w=w, valid=valid, beta=st.beta.copy(), P=st.P.copy(),
                         z=st.z.copy(), rad=rad, mot=mot, var=var, g=g))
    return hist


def _p_vectors(prm, z, g):
    """p = [1, z, g_1..g_n] (Sec. 5.1 with the G-buffer entries of an RLS denoiser)."""
    n = z.shape[0]
    cols = [np.ones((n, 1))]
    if prm.feature_mode == 0:
        cols.append(z)
    if prm.n_gbuf:
        cols.append(g[:prm.n_gbuf].reshape(prm.n_gbuf, n).T.astype(np.float64))
    return np.concatenate(cols, 1)


@pytest.mark.parametrize("kw", [dict(), dict(weight_mode=1), dict(feature_mode=1),
                                dict(init_mode=1, blend_mode=1), dict(radius=0, clamp_mode=1)])
def test_reduces_to_paper_oracle_without_extensions(kw):
    """n_gbuf = 0, Eq. 13 or RLS weight, bilinear reprojection: the extended oracle must
    reproduce the paper-predictor oracle (pinned in test_oracle_pins.py) on a moving
    sequence with restarts."""
    W, H, T = 20, 14, 10
    spec = synth.SceneSpec(W, H, T, seed=21, motion="orbit", firefly_frac=0.05)
    frames = _frames(spec)
    base = O.OracleStream(W, H, O.OracleParams(**kw))
    ext = O.OracleExtStream(W, H, O.OracleExtParams(**kw))
    d = ext.params.dim
    for f in frames:
        rad, mot = f["radiance"].numpy(), f["motion"].numpy()
        o1, w1, v1 = base.frame(rad, mot)
        o2, w2, v2 = ext.frame(rad, mot, f["variance"].numpy(), f["features"].numpy())
        assert np.array_equal(v1, v2)
        assert np.abs(w1 - w2).max() <= 1e-12
        assert np.abs(o1 - o2).max() <= 1e-10 * max(1.0, np.abs(o1).max())
        assert np.abs(base.beta[:, :, :d] - ext.beta).max() <= 1e-10 * max(1.0, np.abs(ext.beta).max())
        assert np.abs(base.P[:, :d, :d] - ext.P).max() <= 1e-10 * max(1.0, np.abs(ext.P).max())


@pytest.mark.parametrize("kw,frames", [(dict(n_gbuf=4), 8), (dict(n_gbuf=4), 60),
                                       (dict(n_gbuf=2, feature_mode=1), 20),
                                       (dict(n_gbuf=3, weight_mode=2), 20),
                                       (dict(n_gbuf=4, init_mode=1), 8)])
def test_recursion_equals_batch_weighted_least_squares_with_gbuffers(kw, frames):
    """Static camera, no restarts after frame 0: P(t)^-1 = lambda^(t+1) P0^-1 +
    sum_s lambda^(t-s) w_s p_s p_s^T and beta_c(t) = P(t)(lambda^(t+1) P0^-1 beta0_c +
    sum_s lambda^(t-s) w_s p_s I~_c,s) with p_s = [1, z_s, g_s] (d up to 8). Uses the z_s
    and w_s of the recursion; checks Eq. 8, 9, 11, 14 in d dimensions and the G-buffer
    entries of p."""
    W = H = 6
    spec = synth.SceneSpec(W, H, frames, seed=22, motion="static", firefly_frac=0.1)
    prm = O.OracleExtParams(**kw)
    hist = _run_ext(_frames(spec), W, H, prm)
    lam, delta, d, n = prm.lambda_, prm.p0_delta, prm.dim, W * H
    beta0 = np.zeros((n, 3, d))
    if prm.init_mode == 1:
        for c in range(3):
            beta0[:, c, c + 1] = 1.0
    A = np.zeros((n, d, d))
    b = np.zeros((n, 3, d))
    for t, h in enumerate(hist):
        p = _p_vectors(prm, h["z"], h["g"])
        w = h["w"].reshape(n)
        I = h["rad"].reshape(3, n).T.astype(np.float64)
        A = lam * A + w[:, None, None] * p[:, :, None] * p[:, None, :]
        b = lam * b + w[:, None, None] * I[:, :, None] * p[:, None, :]
        prior = lam ** (t + 1) / delta
        At = A + prior * np.eye(d)[None]
        bt = b + prior * beta0
        beta_ls = np.linalg.solve(At, bt.transpose(0, 2, 1)).transpose(0, 2, 1)
        P_ls = np.linalg.inv(At)
        assert np.abs(h["beta"] - beta_ls).max() / max(1.0, np.abs(beta_ls).max()) < 1e-8, t
        assert np.abs(h["P"] - P_ls).max() / np.abs(P_ls).max() < 1e-8, t


def test_recursion_equals_bruteforce_stacked_lstsq_d8():
    """Eq. 7 at d = 8: rows sqrt(lambda^(t-s) w_s) [1, z_s, g_s] plus the prior rows,
    solved by QR least squares."""
    W, H, T = 6, 6, 14
    spec = synth.SceneSpec(W, H, T, seed=23, motion="static", firefly_frac=0.05)
    prm = O.OracleExtParams(n_gbuf=4)
    hist = _run_ext(_frames(spec), W, H, prm)
    lam, delta, t = prm.lambda_, prm.p0_delta, T - 1
    for j in range(0, W * H, 5):
        rows, tgt = [], []
        for s in range(t + 1):
            ws = hist[s]["w"].reshape(-1)[j] * lam ** (t - s)
            g = hist[s]["g"].reshape(7, -1)[:4, j].astype(np.float64)
            ps = np.concatenate([[1.0], hist[s]["z"][j], g])
            rows.append(math.sqrt(ws) * ps)
            tgt.append(math.sqrt(ws) * hist[s]["rad"].reshape(3, -1)[:, j].astype(np.float64))
        X = np.vstack(rows + [math.sqrt(lam ** (t + 1) / delta) * np.eye(8)])
        Y = np.vstack(tgt + [np.zeros((8, 3))])
        beta_ls, *_ = np.linalg.lstsq(X, Y, rcond=None)
        assert np.allclose(hist[t]["beta"][j], beta_ls.T, rtol=1e-8, atol=1e-8), j


def test_variance_weight_special_values():
    """Sample-variance weight w = exp(-3 sigma^2 / ((min(|I|,|z|) + eps)^2 h^2)). On a
    restarted pixel z = I~, so the denominator is |I~| + eps: variance 0 gives w = 1, the
    variance that makes the exponent 1 gives 1/e, a negative or non-finite variance gives
    w = 0."""
    W, H = 4, 1
    prm = O.OracleExtParams(weight_mode=2)
    col = np.array([0.3, 0.5, 0.2])
    rad = np.repeat(col[:, None, None], W, 2).astype(np.float32).reshape(3, H, W)
    mot = np.zeros((2, H, W), np.float32)
    nrm = float(np.linalg.norm(rad[:, 0, 0].astype(np.float64))) + prm.eps
    v_e = nrm * nrm * prm.h * prm.h / 3.0
    var = np.array([[0.0, v_e, -1.0, np.nan]], np.float32)
    st = O.OracleExtStream(W, H, prm)
    _, w, _ = st.frame(rad, mot, var)
    expect_e = math.exp(-3.0 * float(np.float32(v_e)) / (nrm * nrm * prm.h * prm.h))
    assert w[0, 0] == 1.0
    assert abs(w[0, 1] - expect_e) < 1e-12 and abs(expect_e - math.exp(-1)) < 1e-6
    assert w[0, 2] == 0.0 and w[0, 3] == 0.0
    # weight 0: beta stays at its restart value (0), P is divided by lambda
    assert np.all(st.beta[2] == 0.0) and np.allclose(st.P[2], np.eye(4) / prm.lambda_, rtol=0, atol=1e-15)


def test_nearest_reprojection_picks_the_rounded_pixel():
    """Nearest-pixel reprojection fetches the model at (floor(qx + 0.5), floor(qy + 0.5)),
    computed in binary32. With the clamp off, Eq. 12 gives
    z_j(1) = alpha z_q(0) + (1 - alpha) I~_j(1) at that pixel exactly; an integer motion
    gives the same state as the bilinear fetch."""
    W, H = 9, 7
    rng = np.random.default_rng(5)
    rad0 = rng.uniform(0.1, 1.0, (3, H, W)).astype(np.float32)
    rad1 = rng.uniform(0.1, 1.0, (3, H, W)).astype(np.float32)
    frac = np.array([0.0, 0.25, 0.5, 0.75, -0.25, -0.5, 1.5, -1.49], np.float32)
    mot = np.stack([rng.choice(frac, (H, W)), rng.choice(frac, (H, W))]).astype(np.float32)
    prm = O.OracleExtParams(reproj_filter=1, clamp_mode=1)
    st = O.OracleExtStream(W, H, prm)
    st.frame(rad0, np.zeros_like(mot))
    z0 = st.z.copy()
    _, _, valid = st.frame(rad1, mot)
    n_checked = 0
    for y in range(H):
        for x in range(W):
            qx = np.float32(x) + mot[0, y, x]
            qy = np.float32(y) + mot[1, y, x]
            ok = 0 <= qx <= W - 1 and 0 <= qy <= H - 1
            assert valid[y, x] == ok
            if not ok:
                continue
            xn = int(math.floor(float(np.float32(qx + np.float32(0.5)))))
            yn = int(math.floor(float(np.float32(qy + np.float32(0.5)))))
            zq = z0[yn * W + xn]
            expect = prm.alpha * zq + (1 - prm.alpha) * rad1[:, y, x].astype(np.float64)
            assert np.allclose(st.z[y * W + x], expect, rtol=0, atol=1e-15), (x, y)
            n_checked += 1
    assert n_checked > W * H // 2
    # integer motion: nearest == bilinear
    mot_i = np.round(mot)
    a = O.OracleExtStream(W, H, O.OracleExtParams(reproj_filter=1))
    b = O.OracleExtStream(W, H, O.OracleExtParams(reproj_filter=0))
    for r, m in ((rad0, np.zeros_like(mot)), (rad1, mot_i), (rad0, mot_i)):
        oa, _, _ = a.frame(r, m)
        ob, _, _ = b.frame(r, m)
        assert np.array_equal(oa, ob) and np.array_equal(a.beta, b.beta) and np.array_equal(a.P, b.P)


def test_nonfinite_gbuffer_value_gives_weight_zero():
    """A non-finite G-buffer value enters p as 0 and the sample gets weight 0: beta stays,
    P is divided by lambda; z is still updated by Eq. 12."""
    W, H = 5, 4
    spec = synth.SceneSpec(W, H, 3, seed=24, motion="static")
    fr = _frames(spec)
    prm = O.OracleExtParams(n_gbuf=2)

    def hook(t, rad, mot, var, g):
        if t == 2:
            g[1, 1, 2] = np.nan
        return rad, mot, var, g
    hist = _run_ext(fr, W, H, prm, hook)
    j = 1 * W + 2
    assert hist[2]["w"][1, 2] == 0.0 and hist[1]["w"][1, 2] > 0.0
    assert np.array_equal(hist[2]["beta"][j], hist[1]["beta"][j])
    assert np.allclose(hist[2]["P"][j], hist[1]["P"][j] / prm.lambda_, rtol=1e-15, atol=0)
    assert np.all(np.isfinite(hist[2]["out"]))
    assert not np.array_equal(hist[2]["z"][j], hist[1]["z"][j])


def test_cross_prediction_uses_the_output_pixels_gbuffer():
    """Blend of a state whose models all read only G-buffer entry 1 (beta_c = e_5): every
    neighbour predicts pixel i as g_1(i), so the normalised cross-prediction blend returns
    g_1(i) exactly; the bilateral average of the neighbours' own predictions returns the
    blend weights' average of g_1 instead (here: not equal to g_1(i))."""
    W, H = 8, 6
    rng = np.random.default_rng(9)
    n = W * H
    z = rng.uniform(0.2, 1.0, (n, 3))
    g = rng.uniform(0.0, 1.0, (4, H, W)).astype(np.float32)
    beta = np.zeros((n, 3, 8))
    beta[:, :, 4] = 1.0
    c = O.lib()
    for blend_mode in (0, 1):
        prm = O.OracleExtParams(n_gbuf=4, blend_mode=blend_mode).c()
        out = np.empty((3, H, W))
        rc = c.wrls_oracle_ext_blend(O.ctypes.byref(prm), W, H, O._dptr(np.ascontiguousarray(beta)),
                                     O._dptr(np.ascontiguousarray(z)), O._fptr(g), O._dptr(out))
        assert rc == 0
        for ch in range(3):
            if blend_mode == 0:
                assert np.allclose(out[ch], g[0], rtol=1e-14, atol=1e-14)
            else:
                assert np.abs(out[ch] - g[0]).max() > 1e-3
