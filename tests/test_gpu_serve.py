"""Serving loop: sessions are admitted as slots free up, their frames join in-flight
batched ticks, and each session's result equals denoising its frames alone."""
import time

import pytest
import torch

from paper_2106_08034_gb300 import serve
from paper_2106_08034_gb300 import wrls as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()
    W.lib()


@pytest.mark.parametrize("precision", [W.WRLS_STATE_BF16, W.WRLS_STATE_F32])
def test_each_session_in_the_mix_equals_alone(precision):
    res = [(64, 48), (96, 64), (128, 72)]
    rings = serve.make_rings(res, frames=3)
    params = W.wrls_params_default(state_precision=precision)
    srv = serve.Server(hbm_budget_bytes=1 << 30, max_sessions=3, params=params, depth=2, rings=rings)
    t0 = time.perf_counter()
    sessions = [serve.Session(i, *res[i % 3], fps=300.0 + 50 * i, arrive=t0 + 0.05 * i, depart=t0 + 100.0)
                for i in range(5)]
    sessions[0].depart = t0 + 0.4           # frees a slot for a queued session
    pending = list(sessions)
    with torch.cuda.stream(srv.cs):
        while time.perf_counter() < t0 + 1.5:
            now = time.perf_counter()
            while pending and pending[0].arrive <= now:
                srv.request(pending.pop(0), now)
            for s in [s for s in srv.active.values() if now >= s.depart and s.in_flight == 0]:
                srv.depart(s.sid, now)
            srv.poll(now)
            if len(srv.ticks) < srv.depth:
                ready = srv.due_frames(now)
                if ready:
                    srv.launch(ready)
    snap = srv.snapshot()
    assert srv.admitted_total >= 4 and srv.max_concurrent == 3
    assert len(snap) == 3 and 0 not in snap
    for sid, (w, h, n, out) in snap.items():
        assert n > 5
        rad, mot = rings[(w, h)]
        alone = W.Stream(w, h, params)
        o = torch.empty(3, h, w, device="cuda")
        for k in range(n):
            alone.denoise(rad[k % rad.shape[0]], mot[k % mot.shape[0]], o)
        torch.cuda.synchronize()
        assert torch.equal(o, out), sid
        alone.close()
    srv.close()
    assert srv.latencies and all(l > 0 for l in srv.latencies)


def test_denoise_batch_entry_equals_per_frame_calls():
    """wrls_denoise_batch (the library's own executor) gives bit for bit the outputs of
    wrls_denoise_frame on each stream, over several ticks of mixed sizes."""
    import torch
    from paper_2106_08034_gb300 import synth
    from paper_2106_08034_gb300 import wrls as W
    sizes = [(96, 64), (160, 90), (72, 40)]
    frames = [[synth.Scene(synth.SceneSpec(w, h, 4, seed=90 + i, motion="orbit", firefly_frac=0.05)).frame(t, device="cuda")
               for t in range(4)] for i, (w, h) in enumerate(sizes)]
    p = W.wrls_params_default(state_precision=W.WRLS_STATE_BF16)
    a = [W.Stream(w, h, p) for w, h in sizes]
    b = [W.Stream(w, h, p) for w, h in sizes]
    oa = [torch.empty(3, h, w, device="cuda") for w, h in sizes]
    ob = [torch.empty(3, h, w, device="cuda") for w, h in sizes]
    for t in range(4):
        W.wrls_denoise_batch([(a[i].handle, frames[i][t]["radiance"], None, None, frames[i][t]["motion"], oa[i])
                              for i in range(len(sizes))])
        for i in range(len(sizes)):
            b[i].denoise(frames[i][t]["radiance"], frames[i][t]["motion"], ob[i])
        torch.cuda.synchronize()
        for i in range(len(sizes)):
            assert torch.equal(oa[i], ob[i]), (t, i)
    for s in a + b:
        s.close()
