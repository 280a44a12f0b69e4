"""The batched tick that allocates nothing (wrls_batch_tick_static), through the C ABI.

Some callers cannot allocate device memory: a plugin inside a host application that owns
the device memory budget, or a frame loop that cannot afford an allocation's implicit
synchronisation. For them the library keeps the batched tick's work table and work
counters in a static device array instead of the cudaMalloc'ed buffers of wrls_batch_create.
This test checks that entry point against the allocating one, bit for bit, on two calls in a
row, with binary32 and BF16 state and with one stream large enough (at least 2^19 pixels)
to run the two-wide blend configuration in the allocating tick; and that it rejects more
frames than its static table holds. It is collected last so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process as well.
"""
import pytest
import torch

from paper_2106_08034_gb300 import synth
from paper_2106_08034_gb300 import wrls as W

from helpers import cpu_frames

pytestmark = pytest.mark.gpu

SIZES = [(200, 120), (64, 48), (1024, 520), (257, 129), (31, 7)]   # 1024 x 520 >= 2^19 pixels


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_08034_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    W.lib()


@pytest.mark.parametrize("precision", [W.WRLS_STATE_F32, W.WRLS_STATE_BF16])
def test_static_tick_matches_allocating_tick_on_two_calls(precision):
    specs = [synth.SceneSpec(w, h, 2, seed=60 + i, motion="orbit", firefly_frac=0.05)
             for i, (w, h) in enumerate(SIZES)]
    frames = [cpu_frames(sp) for sp in specs]
    cs = torch.cuda.Stream()
    p = W.wrls_params_default(state_precision=precision)
    ref_streams = [W.Stream(w, h, p, cuda_stream=cs) for (w, h) in SIZES]
    new_streams = [W.Stream(w, h, p, cuda_stream=cs) for (w, h) in SIZES]
    batch = W.wrls_batch_create(len(SIZES))
    W.wrls_batch_set_cuda_stream(batch, cs)
    try:
        for t in range(2):                       # two calls in a row
            io_ref, io_new, outs_ref, outs_new = [], [], [], []
            for i, (w, h) in enumerate(SIZES):
                rad = frames[i][t]["radiance"].cuda()
                mot = frames[i][t]["motion"].cuda()
                o_ref = torch.full((3, h, w), float("nan"), device="cuda")
                o_new = torch.full((3, h, w), float("nan"), device="cuda")
                io_ref.append((ref_streams[i].handle, rad, None, None, mot, o_ref))
                io_new.append((new_streams[i].handle, rad, None, None, mot, o_new))
                outs_ref.append(o_ref)
                outs_new.append(o_new)
            torch.cuda.synchronize()
            W.wrls_batch_tick(batch, io_ref)
            W.wrls_batch_tick_static(io_new, cs)
            cs.synchronize()
            for o_ref, o_new in zip(outs_ref, outs_new):
                assert torch.isfinite(o_new).all()
                assert torch.equal(o_new, o_ref)
        for s in new_streams:
            W.wrls_stream_check(s.handle)
            assert W.wrls_stream_frames(s.handle) == 2
    finally:
        W.wrls_batch_destroy(batch)
        for s in ref_streams + new_streams:
            s.close()


def test_static_tick_rejects_more_frames_than_its_table_holds():
    n = W.STATIC_BATCH_MAX + 1
    streams = [W.Stream(8, 8) for _ in range(n)]
    buf = torch.zeros(n, 8, 8, 8, device="cuda")
    io = [(streams[k].handle, buf[k, 0:3], None, None, buf[k, 3:5], buf[k, 5:8]) for k in range(n)]
    with pytest.raises(W.WrlsError) as e:
        W.wrls_batch_tick_static(io)
    assert e.value.status == W.WRLS_ERR_INVALID_ARG
    assert "at most %d" % W.STATIC_BATCH_MAX in W.wrls_last_error()
    for s in streams:
        assert W.wrls_stream_frames(s.handle) == 0
        s.close()
