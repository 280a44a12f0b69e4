"""Admission of the serving loop (paper_2106_08034_gb300.serve.Server) on the CPU: session
slots, the device-memory budget (wrls_state_bytes, a host-only call) and the pixel-rate
budget. Stream and batch objects are replaced by fakes, so no GPU is touched."""
import pytest

from paper_2106_08034_gb300 import build as B
from paper_2106_08034_gb300 import serve
from paper_2106_08034_gb300 import wrls as W


class _FakeStream:
    def __init__(self, w, h, params=None, cuda_stream=None):
        self.closed = False
        self.resets = 0

    def close(self):
        self.closed = True

    def reset(self):
        self.resets += 1


@pytest.fixture
def fake_gpu(monkeypatch):
    B.build()
    W.lib()
    monkeypatch.setattr(serve.W, "Stream", _FakeStream)
    monkeypatch.setattr(serve.W, "wrls_batch_create", lambda n: 1)
    monkeypatch.setattr(serve.W, "wrls_batch_set_cuda_stream", lambda b, c: None)


def _server(**kw):
    kw.setdefault("hbm_budget_bytes", 10 ** 12)
    return serve.Server(cuda_stream=object(), device="cpu", **kw)


def test_rate_budget_defers_and_releases(fake_gpu):
    r1080 = 1920 * 1080 * 60.0
    srv = _server(max_sessions=8, rate_budget_px_s=2.5 * r1080)
    for i in range(3):
        srv.request(serve.Session(i, 1920, 1080, 60.0, 0.0, 100.0), 0.0)
    assert sorted(srv.active) == [0, 1] and [s.sid for s in srv.queue] == [2]
    assert srv.waited_rate >= 1 and abs(srv.rate - 2 * r1080) < 1
    # a 720p30 session fits in the half 1080p60 that is left, ahead of the queued 1080p60
    srv.request(serve.Session(3, 1280, 720, 30.0, 0.0, 100.0), 0.0)
    assert 3 in srv.active and [s.sid for s in srv.queue] == [2]
    srv.depart(0, 1.0)
    assert 2 in srv.active and not srv.queue
    assert abs(srv.rate - (2 * r1080 + 1280 * 720 * 30.0)) < 1


def test_memory_budget_and_slots(fake_gpu):
    p = W.wrls_params_default(state_precision=W.WRLS_STATE_BF16)
    one = W.wrls_state_bytes(1920, 1080, p) + 3 * 1920 * 1080 * 4
    srv = _server(hbm_budget_bytes=2 * one + 10, max_sessions=8, params=p)
    for i in range(3):
        srv.request(serve.Session(i, 1920, 1080, 30.0, 0.0, 100.0), 0.0)
    assert len(srv.active) == 2 and srv.rejected_budget >= 1 and srv.used == 2 * one
    srv = _server(max_sessions=2)
    for i in range(3):
        srv.request(serve.Session(i, 640, 360, 30.0, 0.0, 100.0), 0.0)
    assert len(srv.active) == 2 and len(srv.queue) == 1


def test_no_rate_budget_admits_by_memory_only(fake_gpu):
    srv = _server(max_sessions=64)
    for i in range(10):
        srv.request(serve.Session(i, 3840, 2160, 60.0, 0.0, 100.0), 0.0)
    assert len(srv.active) == 10 and srv.waited_rate == 0


def test_tick_coalescing_rule(fake_gpu):
    """A tick starts at once when nothing is in flight; while one is in flight, only once the
    oldest due frame has waited coalesce_s; never beyond `depth` ticks in flight."""
    srv = _server(max_sessions=8, depth=2, coalesce_s=0.002)
    a = serve.Session(0, 640, 360, 60.0, 0.0, 100.0)
    b = serve.Session(1, 640, 360, 60.0, 0.0, 100.0)
    a.next_due, b.next_due = 1.000, 1.0015
    assert not srv.should_launch([], 1.0)
    assert srv.should_launch([a, b], 1.0016)                       # idle GPU: start at once
    srv.ticks.append(serve.Tick(event=None, releases=[], pixels=0))
    assert not srv.should_launch([a, b], 1.0016)                   # busy: oldest waited 1.6 ms
    assert srv.should_launch([a, b], 1.0021)                       # busy: oldest waited 2.1 ms
    srv.ticks.append(serve.Tick(event=None, releases=[], pixels=0))
    assert not srv.should_launch([a, b], 1.0100)                   # depth reached
    srv2 = _server(max_sessions=8, depth=2, coalesce_s=0.0)        # no coalescing window
    srv2.ticks.append(serve.Tick(event=None, releases=[], pixels=0))
    assert srv2.should_launch([a], 1.0)


def test_departed_streams_are_pooled_and_reused(fake_gpu):
    """A departed session's stream is reset and kept for the next session of its resolution
    (no allocation or free in the loop); pooled memory counts against the budget and pooled
    streams are closed when an admission needs the room; at most `pool_per_resolution` are
    kept per resolution."""
    p = W.wrls_params_default(state_precision=W.WRLS_STATE_BF16)
    b1080 = W.wrls_state_bytes(1920, 1080, p) + 3 * 1920 * 1080 * 4
    b4k = W.wrls_state_bytes(3840, 2160, p) + 3 * 3840 * 2160 * 4
    srv = _server(hbm_budget_bytes=b4k + b1080 - 1, max_sessions=8, params=p, pool_per_resolution=1)
    srv.request(serve.Session(0, 1920, 1080, 60.0, 0.0, 100.0), 0.0)
    st0 = srv.active[0].stream
    srv.depart(0, 1.0)
    assert not st0.closed and st0.resets == 1 and srv.pooled == b1080 and srv.used == 0
    srv.request(serve.Session(1, 1920, 1080, 30.0, 1.0, 100.0), 1.0)
    assert srv.active[1].stream is st0 and srv.reused == 1 and srv.pooled == 0 and srv.used == b1080
    srv.request(serve.Session(2, 1920, 1080, 30.0, 1.0, 100.0), 1.0)
    st2 = srv.active[2].stream
    assert st2 is not st0 and srv.used == 2 * b1080
    srv.depart(1, 2.0)
    srv.depart(2, 2.0)            # the pool keeps one stream per resolution: this one is closed
    assert not st0.closed and st2.closed and srv.pooled == b1080
    # a 4K session fits the budget only without the pooled 1080p stream: it is evicted
    srv.request(serve.Session(3, 3840, 2160, 30.0, 3.0, 100.0), 3.0)
    assert 3 in srv.active and st0.closed and srv.pooled == 0 and srv.used == b4k
