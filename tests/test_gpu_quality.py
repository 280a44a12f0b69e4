"""The paper's qualitative claims, on the GPU path, scored against the clean truth
(paper_2106_08034_gb300.quality)."""
import pytest
import torch

from paper_2106_08034_gb300 import quality, synth
from paper_2106_08034_gb300 import wrls as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()
    W.lib()


def test_ablations_follow_the_paper():
    spec = synth.SceneSpec(480, 272, 40, seed=71, motion="orbit", firefly_frac=0.05)
    rep = quality.ablation_report(spec)
    print(rep)
    full = rep["wRLS-F-5x5"]
    assert full["relmse"] < 0.2 * full["relmse_input"]              # Sec. 7.4: improves the input
    assert full["relmse"] < 0.5 * rep["RLS-F-5x5"]["relmse"]         # Fig. 9: wRLS vs RLS on spikes
    assert full["relmse"] < rep["wRLS-F-temporal"]["relmse"]         # Sec. 5.3: the 5x5 blend helps
    assert full["flicker"] < rep["RLS-F-5x5"]["flicker"]


def test_feature_helps_without_spike_noise():
    """Fig. 8: the temporal feature lowers the error. (With 5% x50 fireflies the feature is
    contaminated through its (1 - alpha) share of the sample, and the no-feature model wins on
    relMSE; that case is reported by the bench's quality figures, not asserted.)"""
    spec = synth.SceneSpec(480, 272, 40, seed=73, motion="orbit")
    rep = quality.ablation_report(spec)
    print(rep)
    assert rep["wRLS-F-5x5"]["relmse"] < rep["wRLS-NF-5x5"]["relmse"]


def test_error_falls_with_input_noise():
    """Sec. 7.4 (Fig. 16-17): accuracy improves as the input gets less noisy."""
    spec = synth.SceneSpec(320, 180, 24, seed=72, motion="pan")
    sweep = quality.noise_sweep(spec)
    errs = [sweep[mu]["relmse"] for mu in sorted(sweep)]
    print(sweep)
    assert all(a < b for a, b in zip(errs, errs[1:]))


def test_ablations_on_path_traced_input():
    """The paper's claims on path-traced frames (wrls_render_vpt, 2 spp, reconstruction filter,
    velocities from first collisions), scored against 64-spp renders of the same frames: the
    temporal feature beats a regression on the renderer's noisy G-buffers (Sec. 5.3, Fig. 4,
    8), the Eq. 13 weight beats the sample-variance weight at few samples (Sec. 5.3), the 5x5
    blend lowers the temporal-only error, and the output error is far below the input's."""
    rep = quality.vpt_ablation(width=256, height=144, frames=20)
    print(rep)
    full = rep["wRLS-F-5x5"]
    assert full["relmse"] < 0.5 * full["relmse_input"]
    assert full["relmse"] < 0.85 * rep["RLS-G-5x5"]["relmse"]
    assert full["flicker"] < rep["RLS-G-5x5"]["flicker"]
    assert full["relmse"] < rep["varW-F-5x5"]["relmse"]
    assert full["relmse"] < rep["wRLS-F-temporal"]["relmse"]
    assert full["relmse"] < rep["wRLS-F+G-5x5"]["relmse"]


def test_edits_settle_without_reset():
    """Sec. 5.2: a transfer-function edit and a light move are handled without a reset of the
    models. Reported curve (480 x 272 orbit, no fireflies): the transient after each event
    decays within 10 frames to within 1.5x of the level of the 10 frames after that. (How far
    that level sits above the pre-edit error is reported, not gated: after the palette remap
    the models re-fit at the rate lambda and P allow.)"""
    rep = quality.edit_recovery()
    print(rep["events"])
    assert set(rep["events"]) == {"tf_edit", "light_move"}
    for ev in rep["events"].values():
        assert ev["frames_to_settle"] is not None and ev["frames_to_settle"] <= 10, ev


def test_runtime_depends_on_resolution_only():
    """Sec. 7: the cost per frame depends on the resolution, not on the content or the motion:
    equal-size sequences of different content and motion (static, pan, orbit) take the same
    kernel time within 15 %."""
    rep = quality.runtime_vs_content(sizes=((960, 540),), seeds=(5, 6), frames=8)
    print(rep)
    assert rep["960x540"]["spread"] < 1.15
