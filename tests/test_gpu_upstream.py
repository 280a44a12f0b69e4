"""Parity of the CUDA input steps (pixel reconstruction filter, velocity from first-collision
world positions) with the FP64 oracle (oracle/wrls_oracle_upstream.c), through the C ABI,
and of the whole chain raw samples -> reconstruction -> velocity -> denoiser."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import REL_TOL, oracle_params_from, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    W.lib()


def _rel_close(a, b, tol=REL_TOL, floor=1e-12):
    """Elementwise relative closeness with identical non-finite positions."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb), "non-finite positions differ"
    err = np.abs(a[fa] - b[fa]) / np.maximum(np.abs(b[fa]), floor)
    return float(err.max()) if err.size else 0.0


@pytest.mark.parametrize("spp,sigma,radius,size", [(1, 0.5, 1.5, (97, 61)), (2, 0.5, 1.5, (250, 130)),
                                                   (4, 0.8, 0.9, (64, 40)), (8, 0.35, 1.5, (33, 17))])
def test_reconstruction_matches_oracle(spp, sigma, radius, size):
    W_, H_ = size
    sc = synth.Scene(synth.SceneSpec(W_, H_, 2, seed=81 + spp, motion="pan", firefly_frac=0.05))
    smp = synth.raw_samples(sc, 1, spp)
    smp[0, 1, 3, 4] = float("nan")          # missing colour
    smp[spp - 1, 3, 5, 6] = float("inf")    # missing offset
    smp[:, 0, 0, 0] = float("nan")          # a pixel without any valid sample
    p = W.wrls_recon_params_default(sigma=sigma, radius=radius)
    d = smp.cuda()
    rad = torch.empty(3, H_, W_, device="cuda")
    var = torch.empty(H_, W_, device="cuda")
    W.wrls_reconstruct(d, rad, var, p)
    torch.cuda.synchronize()
    ref, rvar = O.reconstruct(smp.numpy(), sigma=sigma, radius=radius)
    assert rel_err(rad.cpu().numpy(), ref) <= REL_TOL
    assert _rel_close(var.cpu().numpy(), rvar) <= REL_TOL
    W.wrls_reconstruct(d, rad, None, p)       # variance output is optional
    torch.cuda.synchronize()
    assert rel_err(rad.cpu().numpy(), ref) <= REL_TOL


def test_velocity_matches_oracle_full_hd():
    W_, H_ = 1920, 1080
    M_prev = synth.orbit_camera(9, W_, H_)
    world = synth.first_collision_world(W_, H_, synth.orbit_camera(10, W_, H_), seed=3)
    d = torch.from_numpy(world).cuda()
    for policy in (0, 1):
        mot = torch.empty(2, H_, W_, device="cuda")
        W.wrls_velocity_from_world(d, M_prev, mot, miss_policy=policy)
        torch.cuda.synchronize()
        ref = O.velocity(world, M_prev.astype(np.float32).astype(np.float64), policy)
        got = mot.cpu().numpy()
        fin = np.isfinite(ref)
        assert np.array_equal(fin, np.isfinite(got))
        assert np.abs(got[fin] - ref[fin]).max() <= 2e-3      # pixels
        assert np.abs(ref[fin]).max() > 1.0                   # the camera did move


def test_chain_samples_to_denoised_output():
    """Raw samples -> reconstruction -> velocity -> denoiser on the GPU, against the same
    chain of oracles fed with their own intermediate results (binary32 between the steps)."""
    W_, H_, T = 160, 96, 8
    spec = synth.SceneSpec(W_, H_, T, seed=85, motion="static", firefly_frac=0.02)
    sc = synth.Scene(spec)
    s = W.Stream(W_, H_)
    st = O.OracleStream(W_, H_, oracle_params_from(W.wrls_params_default()))
    rad = torch.empty(3, H_, W_, device="cuda")
    mot = torch.empty(2, H_, W_, device="cuda")
    out = torch.empty(3, H_, W_, device="cuda")
    for t in range(T):
        smp = synth.raw_samples(sc, t, 2)
        world = synth.first_collision_world(W_, H_, synth.orbit_camera(t, W_, H_), seed=t)
        M_prev = synth.orbit_camera(t - 1, W_, H_)
        W.wrls_reconstruct(smp.cuda(), rad)
        W.wrls_velocity_from_world(torch.from_numpy(world).cuda(), M_prev, mot)
        s.denoise(rad, mot, out)
        torch.cuda.synchronize()
        r_rad, _ = O.reconstruct(smp.numpy(), with_variance=False)
        r_mot = O.velocity(world, M_prev.astype(np.float32).astype(np.float64))
        ref, _, _ = st.frame(r_rad.astype(np.float32), r_mot.astype(np.float32))
        assert rel_err(out.cpu().numpy(), ref) <= REL_TOL, t
    s.close()


def test_input_steps_reject_bad_arguments():
    x = torch.zeros(1, 5, 8, 8, device="cuda")
    r = torch.empty(3, 8, 8, device="cuda")
    with pytest.raises(W.WrlsError):
        W.wrls_reconstruct(x, r, params=W.wrls_recon_params_default(radius=2.0))
    with pytest.raises(W.WrlsError):
        W.wrls_reconstruct(x, x[0, :3])              # output overlaps the samples
    with pytest.raises(W.WrlsError):
        W.wrls_velocity_from_world(r, np.full((4, 4), np.nan), torch.empty(2, 8, 8, device="cuda"))
