"""Seeded synthetic frame sequences that stand in for the paper's 2-spp volumetric
path-traced frames (the Table 3 volumes and the 1024-spp references are not available).

This module holds none of the denoiser's arithmetic. It only produces, per frame,
the inputs of the per-frame denoising problem of Sec. 4 / Fig. 5 and the clean truth:

* ``truth``     (3, H, W) f32: smooth procedural shading (Lambert of a seeded
  low-frequency height field) times a smooth albedo, overlaid by 20-60 random
  hard-edged discs, clipped to [0, 1].
* ``radiance``  (3, H, W) f32: truth + N(0, s^2) per channel, with
  ln s^2 ~ N(mu, sigma^2) drawn per pixel per frame (heteroscedastic in time);
  optionally a fraction of pixels are fireflies (value x gain).
* ``variance``  (H, W) f32: the s^2 that was drawn.
* ``features``  (7, H, W) f32: depth, normal (3), albedo (3), clean values plus
  noise at ``feature_noise_rel`` x the radiance std (the noisy G-buffers of Fig. 4).
* ``motion``    (2, H, W) f32: backward motion in pixels, planar (vx, vy), with
  the previous-frame position of pixel j being j + v_j (Table 2, pi(v_j)).

Scene content is evaluated at continuous scene coordinates u = M_t(x) of each pixel
centre x, so camera motion is exact: static (M_t = id), pan (u = x + t * pan), or an
orbit (rotation + zoom + drift about the image centre). Optional events: a transfer
function edit (albedo remap) and a light move (azimuth + 30 deg).

Random numbers come from ``torch.Generator`` seeded per (scene seed, frame), so a
sequence is reproducible on one device type; CPU and CUDA draws differ. Parity tests
generate on the CPU and copy the same arrays to the GPU.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

N_FEATURES = 7


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    width: int
    height: int
    frames: int
    seed: int = 0
    motion: str = "static"          # "static" | "pan" | "orbit"
    pan_px: float = 1.7             # pan speed in px/frame along +x of the scene
    noise_mu: float = -4.0          # ln variance mean
    noise_sigma: float = 1.5        # ln variance std
    firefly_frac: float = 0.0       # fraction of pixels per frame scaled by firefly_gain
    firefly_gain: float = 50.0
    feature_noise_rel: float = 0.3
    tf_edit_frame: Optional[int] = None
    light_move_frame: Optional[int] = None
    noiseless: bool = False         # radiance == truth (zero-noise checks)

    @property
    def pixels(self) -> int:
        return self.width * self.height


# --- named workloads --------------------------------------------------------------

def static_128x128_8f(seed: int = 0) -> SceneSpec:
    """128x128, 8 frames, static camera, heteroscedastic log-normal noise, no fireflies."""
    return SceneSpec(128, 128, 8, seed=seed, motion="static")


def pan_1080p_120f(seed: int = 1) -> SceneSpec:
    """1920x1080, 120 frames, camera pan of 1.7 px/frame, 5% fireflies (x50)."""
    return SceneSpec(1920, 1080, 120, seed=seed, motion="pan", pan_px=1.7,
                     firefly_frac=0.05)


def orbit_edit_1080p_120f(seed: int = 2) -> SceneSpec:
    """1920x1080, 120 frames, seeded affine camera orbit, transfer-function edit at
    frame 60 and a 30-degree light move at frame 90, 5% fireflies."""
    return SceneSpec(1920, 1080, 120, seed=seed, motion="orbit", firefly_frac=0.05,
                     tf_edit_frame=60, light_move_frame=90)


MIX16_SIZES = ([(512, 512)] * 4 + [(1280, 720)] * 4 + [(1920, 1080)] * 4 +
               [(2560, 1440)] * 2 + [(3840, 2160)] * 2)


def mix16_60f(seed: int = 3, frames: int = 60) -> List[SceneSpec]:
    """16 concurrent streams of mixed sizes (4x512^2, 4x720p, 4x1080p, 2x1440p,
    2x2160p), 60 frames each, independent seeds and orbit motion."""
    return [SceneSpec(w, h, frames, seed=seed * 1000 + i, motion="orbit", firefly_frac=0.05)
            for i, (w, h) in enumerate(MIX16_SIZES)]


SERVING_RESOLUTIONS = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]


# --- scene ---------------------------------------------------------------------------

class Scene:
    """A seeded procedural scene; ``frame(t)`` renders frame t on a torch device."""

    def __init__(self, spec: SceneSpec):
        self.spec = spec
        rng = np.random.default_rng(np.random.PCG64(spec.seed + 7919))
        W, H = spec.width, spec.height
        S = float(H)
        self.S = S
        # height field: 4 low-frequency sines, slopes O(1)
        nh = 4
        ang = rng.uniform(0, 2 * math.pi, nh)
        cyc = rng.uniform(0.5, 2.5, nh)                      # cycles per S
        self.h_f = np.stack([np.cos(ang), np.sin(ang)], 1) * (2 * math.pi * cyc / S)[:, None]
        self.h_phase = rng.uniform(0, 2 * math.pi, nh)
        slope = rng.uniform(0.3, 0.8, nh) / 2.0
        self.h_amp = slope / (2 * math.pi * cyc / S)         # gradient amplitude = slope
        # light
        self.l_theta = math.radians(50.0)
        self.l_phi = rng.uniform(0, 2 * math.pi)
        # smooth albedo per channel
        a_ang = rng.uniform(0, 2 * math.pi, 3)
        a_cyc = rng.uniform(0.3, 1.5, 3)
        self.a_f = np.stack([np.cos(a_ang), np.sin(a_ang)], 1) * (2 * math.pi * a_cyc / S)[:, None]
        self.a_phase = rng.uniform(0, 2 * math.pi, 3)
        # camera
        self.orbit_w = math.radians(rng.uniform(0.15, 0.35)) * (1 if rng.random() < 0.5 else -1)
        self.orbit_zoom = rng.uniform(-1e-3, 1e-3)
        self.orbit_drift = rng.uniform(-0.8, 0.8, 2)
        self.centre = np.array([(W - 1) / 2.0, (H - 1) / 2.0])
        # discs over the region the camera will see
        nd = int(rng.integers(20, 61))
        if spec.motion == "pan":
            x_lo, x_hi = -0.1 * W, 1.1 * W + spec.pan_px * spec.frames
            y_lo, y_hi = -0.1 * H, 1.1 * H
        elif spec.motion == "orbit":
            R = 0.75 * math.hypot(W, H) + float(np.abs(self.orbit_drift).max()) * spec.frames
            x_lo, x_hi = self.centre[0] - R, self.centre[0] + R
            y_lo, y_hi = self.centre[1] - R, self.centre[1] + R
        else:
            x_lo, x_hi, y_lo, y_hi = -0.1 * W, 1.1 * W, -0.1 * H, 1.1 * H
        area_scale = max(1.0, (x_hi - x_lo) * (y_hi - y_lo) / (1.2 * W * 1.2 * H))
        nd = int(min(4 * nd, round(nd * area_scale)))
        self.d_c = np.stack([rng.uniform(x_lo, x_hi, nd), rng.uniform(y_lo, y_hi, nd)], 1)
        self.d_r = rng.uniform(0.03, 0.09, nd) * S
        self.d_col = rng.uniform(0.05, 0.95, (nd, 3))

    # camera map u = centre + A_t (x - centre) + b_t, A_t a similarity
    def _camera(self, t: int):
        sp = self.spec
        if sp.motion == "pan":
            return 1.0, 0.0, np.array([sp.pan_px * t, 0.0])
        if sp.motion == "orbit":
            return 1.0 + self.orbit_zoom * t, self.orbit_w * t, self.orbit_drift * t
        return 1.0, 0.0, np.zeros(2)

    def _coords(self, t: int, device):
        W, H = self.spec.width, self.spec.height
        s, th, b = self._camera(t)
        xs = torch.arange(W, dtype=torch.float64, device=device)
        ys = torch.arange(H, dtype=torch.float64, device=device)
        X = xs[None, :].expand(H, W) - self.centre[0]
        Y = ys[:, None].expand(H, W) - self.centre[1]
        c, sn = math.cos(th), math.sin(th)
        u = self.centre[0] + s * (c * X - sn * Y) + b[0]
        v = self.centre[1] + s * (sn * X + c * Y) + b[1]
        return u, v

    def motion(self, t: int, device="cpu") -> torch.Tensor:
        """Backward motion v_j with previous position j + v_j, (2, H, W) f32."""
        W, H = self.spec.width, self.spec.height
        if t == 0 or self.spec.motion == "static":
            return torch.zeros(2, H, W, dtype=torch.float32, device=device)
        if self.spec.motion == "pan":
            out = torch.zeros(2, H, W, dtype=torch.float32, device=device)
            out[0] = float(np.float32(self.spec.pan_px))
            return out
        u, v = self._coords(t, device)
        s0, th0, b0 = self._camera(t - 1)
        du, dv = u - self.centre[0] - b0[0], v - self.centre[1] - b0[1]
        c, sn = math.cos(-th0), math.sin(-th0)
        xp = self.centre[0] + (c * du - sn * dv) / s0
        yp = self.centre[1] + (sn * du + c * dv) / s0
        xs = torch.arange(W, dtype=torch.float64, device=device)[None, :]
        ys = torch.arange(H, dtype=torch.float64, device=device)[:, None]
        return torch.stack([xp - xs, yp - ys]).to(torch.float32)

    def _clean(self, t: int, device):
        sp = self.spec
        W, H = sp.width, sp.height
        u64, v64 = self._coords(t, device)
        u, v = u64.to(torch.float32), v64.to(torch.float32)
        # height field and its gradient
        hgt = torch.zeros_like(u)
        gx = torch.zeros_like(u)
        gy = torch.zeros_like(u)
        for k in range(len(self.h_amp)):
            ph = (u64 * self.h_f[k, 0] + v64 * self.h_f[k, 1] + self.h_phase[k]).to(torch.float32)
            a = float(self.h_amp[k])
            hgt += a * torch.sin(ph)
            cph = torch.cos(ph)
            gx += (a * float(self.h_f[k, 0])) * cph
            gy += (a * float(self.h_f[k, 1])) * cph
        nrm = torch.rsqrt(gx * gx + gy * gy + 1.0)
        n = torch.stack([-gx * nrm, -gy * nrm, nrm])
        phi = self.l_phi
        if sp.light_move_frame is not None and t >= sp.light_move_frame:
            phi += math.radians(30.0)
        L = (math.sin(self.l_theta) * math.cos(phi), math.sin(self.l_theta) * math.sin(phi),
             math.cos(self.l_theta))
        ndl = (n[0] * L[0] + n[1] * L[1] + n[2] * L[2]).clamp_min(0.0)
        shade = 0.2 + 0.8 * ndl
        alb = torch.stack([
            0.5 + 0.3 * torch.sin((u64 * self.a_f[c, 0] + v64 * self.a_f[c, 1]
                                   + self.a_phase[c]).to(torch.float32))
            for c in range(3)])
        # hard-edged discs (later discs on top), evaluated only inside their boxes
        s, th, b = self._camera(t)
        cth, sth = math.cos(-th), math.sin(-th)
        for k in range(len(self.d_r)):
            dc = self.d_c[k] - self.centre - b
            xc = self.centre[0] + (cth * dc[0] - sth * dc[1]) / s
            yc = self.centre[1] + (sth * dc[0] + cth * dc[1]) / s
            rr = self.d_r[k] / s + 2.0
            x0, x1 = max(0, int(math.floor(xc - rr))), min(W, int(math.ceil(xc + rr)) + 1)
            y0, y1 = max(0, int(math.floor(yc - rr))), min(H, int(math.ceil(yc + rr)) + 1)
            if x0 >= x1 or y0 >= y1:
                continue
            du = u64[y0:y1, x0:x1] - self.d_c[k, 0]
            dv = v64[y0:y1, x0:x1] - self.d_c[k, 1]
            inside = (du * du + dv * dv) <= self.d_r[k] ** 2
            for c in range(3):
                blk = alb[c, y0:y1, x0:x1]
                blk[inside] = float(self.d_col[k, c])
        if sp.tf_edit_frame is not None and t >= sp.tf_edit_frame:
            alb = torch.stack([alb[1], alb[2], alb[0]]).pow(1.5)
        truth = (alb * shade[None]).clamp(0.0, 1.0)
        depth = 0.5 + 0.5 * hgt / float(np.abs(self.h_amp).sum())
        feats = torch.cat([depth[None], n, alb], 0)
        return truth, feats

    def frame(self, t: int, device="cpu") -> Dict[str, torch.Tensor]:
        sp = self.spec
        H, W = sp.height, sp.width
        truth, feats = self._clean(t, device)
        gen = torch.Generator(device=device)
        gen.manual_seed((sp.seed * 1_000_003 + t * 7919 + 12345) & 0x7FFFFFFFFFFF)
        g_var = torch.randn(H, W, generator=gen, device=device, dtype=torch.float32)
        var = torch.exp(sp.noise_mu + sp.noise_sigma * g_var)
        std = torch.sqrt(var)
        g_rad = torch.randn(3, H, W, generator=gen, device=device, dtype=torch.float32)
        g_feat = torch.randn(N_FEATURES, H, W, generator=gen, device=device, dtype=torch.float32)
        u_ff = torch.rand(H, W, generator=gen, device=device, dtype=torch.float32)
        if sp.noiseless:
            rad = truth.clone()
        else:
            rad = truth + std[None] * g_rad
            if sp.firefly_frac > 0:
                rad = torch.where((u_ff < sp.firefly_frac)[None], rad * sp.firefly_gain, rad)
        feats_noisy = feats + (sp.feature_noise_rel * std)[None] * g_feat
        return {
            "truth": truth.contiguous(),
            "radiance": rad.contiguous(),
            "variance": var.contiguous(),
            "features": feats_noisy.contiguous(),
            "motion": self.motion(t, device).contiguous(),
        }

    def frames(self, device="cpu", keys: Sequence[str] = ("radiance", "motion", "truth"),
               count: Optional[int] = None) -> Dict[str, torch.Tensor]:
        """All frames stacked along a new leading axis (T, C, H, W) for the given keys."""
        T = self.spec.frames if count is None else count
        acc: Dict[str, list] = {k: [] for k in keys}
        for t in range(T):
            f = self.frame(t, device)
            for k in keys:
                acc[k].append(f[k])
        return {k: torch.stack(v) for k, v in acc.items()}


# ---- raw samples and camera geometry (inputs of the reconstruction and velocity steps) ----

def raw_samples(scene: "Scene", t: int, spp: int, device="cpu") -> torch.Tensor:
    """spp light-path samples per pixel of frame t: (spp, 5, H, W) f32 planes r, g, b, ox, oy.
    Offsets uniform in [-0.5, 0.5) from the pixel centre; each sample is the pixel's clean
    colour plus Gaussian noise of variance spp * sigma_j^2 (so the pixel mean has the frame's
    variance sigma_j^2), times the firefly gain with the scene's firefly probability."""
    sp = scene.spec
    H, W = sp.height, sp.width
    truth, _ = scene._clean(t, device)
    gen = torch.Generator(device=device)
    gen.manual_seed((sp.seed * 2_000_003 + t * 104_729 + spp * 31 + 777) & 0x7FFFFFFFFFFF)
    g_var = torch.randn(H, W, generator=gen, device=device, dtype=torch.float32)
    var = torch.exp(sp.noise_mu + sp.noise_sigma * g_var)
    out = torch.empty(spp, 5, H, W, device=device, dtype=torch.float32)
    for s in range(spp):
        noise = torch.randn(3, H, W, generator=gen, device=device, dtype=torch.float32)
        col = truth + torch.sqrt(var * spp)[None] * noise
        if sp.firefly_frac > 0 and not sp.noiseless:
            u = torch.rand(H, W, generator=gen, device=device, dtype=torch.float32)
            col = torch.where((u < sp.firefly_frac)[None], col * sp.firefly_gain, col)
        if sp.noiseless:
            col = truth.clone()
        out[s, 0:3] = col
        out[s, 3:5] = torch.rand(2, H, W, generator=gen, device=device, dtype=torch.float32) - 0.5
    return out


def perspective_view_proj(eye, target, fov_y_deg: float, aspect: float, near: float = 0.1,
                          far: float = 100.0) -> np.ndarray:
    """Row-major 4x4 view-projection matrix (right-handed view, OpenGL-style clip space)."""
    eye, target = np.asarray(eye, np.float64), np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = r, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    k = 1.0 / math.tan(math.radians(fov_y_deg) / 2)
    proj = np.zeros((4, 4))
    proj[0, 0], proj[1, 1] = k / aspect, k
    proj[2, 2], proj[2, 3] = (far + near) / (near - far), 2 * far * near / (near - far)
    proj[3, 2] = -1.0
    return proj @ view


def orbit_camera(t: int, width: int, height: int, deg_per_frame: float = 0.5) -> np.ndarray:
    """View-projection of frame t of a camera orbiting the origin at radius 4, 45 deg fov."""
    a = math.radians(30.0 + deg_per_frame * t)
    eye = (4.0 * math.sin(a), 1.5, 4.0 * math.cos(a))
    return perspective_view_proj(eye, (0.0, 0.0, 0.0), 45.0, width / height)


def first_collision_world(width: int, height: int, view_proj: np.ndarray, seed: int = 0,
                          miss_frac: float = 0.1) -> np.ndarray:
    """World positions (3, H, W) f32 of points seen through the pixel centres of a camera:
    each pixel's ray (through its centre) is cut at a smooth pseudo-random depth (NDC z in
    [0.90, 0.98]); a seeded `miss_frac` of pixels (blobs) have no collision (NaN)."""
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    ndc_x = (xs + 0.5) / width * 2 - 1
    ndc_y = 1 - (ys + 0.5) / height * 2
    ph = rng.uniform(0, 2 * np.pi, 4)
    zn = 0.94 + 0.04 * np.sin(xs / width * 6.0 + ph[0]) * np.cos(ys / height * 5.0 + ph[1])
    clip = np.stack([ndc_x, ndc_y, zn, np.ones_like(zn)], 0).reshape(4, -1)
    X = np.linalg.inv(view_proj) @ clip
    X = (X[:3] / X[3]).reshape(3, height, width)
    blob = np.sin(xs / width * 9.0 + ph[2]) * np.sin(ys / height * 7.0 + ph[3])
    X[:, blob > np.quantile(blob, 1 - miss_frac)] = np.nan
    return X.astype(np.float32)


# ---- procedural volume scene for the path tracer (parameters only) ----

def vpt_scene(width: int, height: int, t: int = 0, seed: int = 0, n_blobs: int = 12, mu_max: float = 6.0,
              albedo: float = 0.9, max_bounces: int = 4, tf_edit_frame: Optional[int] = None,
              light_move_frame: Optional[int] = None, deg_per_frame: float = 0.5) -> dict:
    """Parameters of frame t of a seeded procedural volume scene: Gaussian density blobs in
    [-1, 1]^3, an opacity ramp and a colour ramp (the transfer function), a directional light
    and an environment, and the orbit camera of `orbit_camera` (eye and inverse
    view-projection). A transfer-function edit swaps the colour ramp and lowers the opacity
    ramp from `tf_edit_frame` on; the light turns by 60 degrees from `light_move_frame` on."""
    rng = np.random.default_rng(seed)
    blobs = np.zeros((16, 5), np.float32)
    for i in range(n_blobs):
        blobs[i, :3] = rng.uniform(-0.55, 0.55, 3)
        blobs[i, 3] = rng.uniform(0.18, 0.42)
        blobs[i, 4] = rng.uniform(0.5, 1.2)
    vp = orbit_camera(t, width, height, deg_per_frame)
    a = math.radians(30.0 + deg_per_frame * t)
    eye = np.array([4.0 * math.sin(a), 1.5, 4.0 * math.cos(a)], np.float32)
    edited = tf_edit_frame is not None and t >= tf_edit_frame
    moved = light_move_frame is not None and t >= light_move_frame
    la = math.radians(-40.0 + (60.0 if moved else 0.0))
    light = np.array([math.cos(la) * 0.6, 0.8, math.sin(la) * 0.6], np.float64)
    light /= np.linalg.norm(light)
    return {
        "seed": (seed * 2654435761 + 12345) & 0xFFFFFFFF, "seed_hi": 0x5EED0000 + seed,
        "eye": eye, "inv_view_proj": np.linalg.inv(vp).astype(np.float32),
        "n_blobs": n_blobs, "blobs": blobs, "mu_max": float(mu_max),
        "tf_lo": 0.05 if not edited else 0.02, "tf_hi": 0.6 if not edited else 0.4, "albedo": float(albedo),
        "color_lo": np.array([0.9, 0.5, 0.3] if not edited else [0.3, 0.6, 0.9], np.float32),
        "color_hi": np.array([1.0, 0.95, 0.85] if not edited else [0.85, 1.0, 0.9], np.float32),
        "light_dir": light.astype(np.float32), "light_rgb": np.array([12.0, 11.0, 10.0], np.float32),
        "env_rgb": np.array([0.25, 0.3, 0.4], np.float32), "max_bounces": int(max_bounces),
    }
