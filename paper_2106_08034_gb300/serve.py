"""Serving loop for interactive viewer sessions (continuous batching over the C ABI).

A session is one viewer: a resolution, a frame rate and a lifetime. It is admitted when a
session slot is free, the device memory its persistent per-pixel state needs
(``wrls_state_bytes``) plus its output buffer fits the memory budget, and (when a rate
budget is set) the pixel rate of the admitted sessions plus its own width x height x fps
stays within the rate budget -- a fraction of the throughput the GPU sustains, so that
frames keep their deadline instead of queueing on the device; otherwise it waits in the
queue until a departure frees room. Admitted sessions keep their state resident on the
device across frames. A departed session's stream (state and output buffer) is reset and kept
in a per-resolution pool for the next session of that resolution, so that admission and
departure make no device allocation or free in the loop (a free waits for the device); pooled
memory counts against the budget and pooled streams are closed when an admission needs the
room. A reset stream restarts every pixel on its next frame, as a new one does, so a
session's output does not depend on whether its stream was pooled.

A tick takes every session whose next frame is due and denoises all of them with one
``wrls_batch_tick``: one CUDA graph launch that holds each session's own update and blend
kernels on four parallel branches, so that one session's blend runs beside another's update.
Up to ``depth`` ticks are in flight; a tick starts as soon as fewer are, so frames that fall
due while the GPU is busy gather into the next tick and ticks grow with the load (continuous
batching). With ``coalesce_s`` > 0 a tick that would start while another is in flight waits
until the oldest due frame has waited that long; measured, that only adds latency (larger
ticks ran no faster per pixel), so it is off by default. Sessions that arrive while others
are on the GPU join the next tick and their work overlaps on the device.

A frame's latency is the time from its release (its due time) to the completion of the tick
that denoised it, observed on the host by polling the tick's CUDA event. If a session falls
more than one frame behind, the older due frames are dropped.

Inputs come from per-resolution rings of pre-generated frames on the device (frames 1..K of a
seeded orbit sequence, all with camera motion), read-only and shared by sessions of one
resolution; session k's n-th processed frame is ring[n % len].
"""
from __future__ import annotations

import dataclasses
import heapq
import math
import random
import time
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import synth
from . import wrls as W


@dataclasses.dataclass
class Session:
    sid: int
    width: int
    height: int
    fps: float
    arrive: float
    depart: float
    stream: Optional[W.Stream] = None
    out: Optional[torch.Tensor] = None
    bytes: int = 0
    next_due: float = 0.0
    processed: int = 0
    dropped: int = 0
    in_flight: int = 0


@dataclasses.dataclass
class Tick:
    event: torch.cuda.Event
    releases: List[Tuple[int, float]]   # (sid, release time) per frame
    pixels: int
    start: Optional[torch.cuda.Event] = None


class Server:
    """Admission by device memory, continuous batching, latency accounting."""

    def __init__(self, hbm_budget_bytes: int, max_sessions: int = 64,
                 params: Optional[W.wrls_params] = None, depth: int = 2, deadline_s: float = 1 / 60,
                 rings: Optional[Dict[Tuple[int, int], Tuple[torch.Tensor, torch.Tensor]]] = None,
                 cuda_stream: Optional[torch.cuda.Stream] = None, rate_budget_px_s: Optional[float] = None,
                 device="cuda", coalesce_s: float = 0.0, pool_per_resolution: int = 4):
        self.budget = int(hbm_budget_bytes)
        self.rate_budget = None if rate_budget_px_s is None else float(rate_budget_px_s)
        self.rate = 0.0              # pixel rate (px/s) of the admitted sessions
        self.device = device
        self.max_sessions = int(max_sessions)
        self.params = params if params is not None else W.wrls_params_default(state_precision=W.WRLS_STATE_BF16)
        self.depth = int(depth)
        self.coalesce = float(coalesce_s)
        self.deadline = float(deadline_s)
        self.rings = rings if rings is not None else {}
        self.cs = cuda_stream if cuda_stream is not None else torch.cuda.Stream()
        self.batch = W.wrls_batch_create(self.max_sessions)
        W.wrls_batch_set_cuda_stream(self.batch, self.cs)
        self.active: Dict[int, Session] = {}
        self.queue: List[Session] = []
        self.used = 0                # bytes of the active sessions
        self.pool: Dict[Tuple[int, int], List[Tuple[W.Stream, torch.Tensor]]] = {}
        self.pooled = 0              # bytes of the pooled streams
        self.pool_max = int(pool_per_resolution)
        self.reused = 0              # admissions served from the pool
        self.ticks: List[Tick] = []
        self.latencies: List[float] = []
        self.missed = 0
        self.frames_done = 0
        self.pixels_done = 0
        self.gpu_ms = 0.0            # device time of the completed ticks (CUDA events)
        self.ticks_done = 0
        self.admitted_total = 0
        self.max_concurrent = 0
        self.rejected_budget = 0
        self.waited_rate = 0         # admission attempts deferred by the rate budget

    # --- admission --------------------------------------------------------------------
    def session_bytes(self, w: int, h: int) -> int:
        return W.wrls_state_bytes(w, h, self.params) + 3 * w * h * 4

    def request(self, s: Session, now: float) -> None:
        self.queue.append(s)
        self._admit(now)

    def _admit(self, now: float) -> None:
        keep = []
        for s in self.queue:
            need = self.session_bytes(s.width, s.height)
            rate = s.width * s.height * s.fps
            rate_ok = self.rate_budget is None or self.rate + rate <= self.rate_budget
            if len(self.active) < self.max_sessions and self.used + need <= self.budget and rate_ok:
                s.bytes = need
                pooled = self.pool.get((s.width, s.height))
                if pooled:
                    s.stream, s.out = pooled.pop()
                    self.pooled -= need
                    self.reused += 1
                else:
                    self._evict(self.budget - self.used - need)
                    s.stream = W.Stream(s.width, s.height, self.params, cuda_stream=self.cs)
                    s.out = torch.empty(3, s.height, s.width, device=self.device)
                s.next_due = max(now, s.arrive)
                self.active[s.sid] = s
                self.used += need
                self.rate += rate
                self.admitted_total += 1
            else:
                if self.used + need > self.budget:
                    self.rejected_budget += 1
                if not rate_ok:
                    self.waited_rate += 1
                keep.append(s)
        self.queue = keep
        self.max_concurrent = max(self.max_concurrent, len(self.active))

    def depart(self, sid: int, now: float) -> None:
        s = self.active.get(sid)
        if s is None:
            self.queue = [q for q in self.queue if q.sid != sid]
            return
        if s.in_flight:
            s.depart = now      # leave after its frames complete
            return
        del self.active[sid]
        self.used -= s.bytes
        self.rate -= s.width * s.height * s.fps
        pooled = self.pool.setdefault((s.width, s.height), [])
        if len(pooled) < self.pool_max:
            s.stream.reset()          # the next session starts from a restart of every pixel
            pooled.append((s.stream, s.out))
            self.pooled += s.bytes
        else:
            s.stream.close()
        s.stream, s.out = None, None
        self._admit(now)

    def _evict(self, room: int) -> None:
        """Close pooled streams, largest first, until they hold at most `room` bytes."""
        while self.pooled > max(room, 0) and any(self.pool.values()):
            key = max((k for k, v in self.pool.items() if v), key=lambda k: k[0] * k[1])
            stream, _ = self.pool[key].pop()
            stream.close()
            self.pooled -= self.session_bytes(*key)

    # --- batching ---------------------------------------------------------------------
    def due_frames(self, now: float) -> List[Session]:
        ready = []
        for s in self.active.values():
            if s.in_flight or now < s.next_due or now >= s.depart:
                continue
            period = 1.0 / s.fps
            behind = int((now - s.next_due) / period)
            if behind > 0:                      # keep only the newest due frame
                s.dropped += behind
                self.missed += behind
                s.next_due += behind * period
            ready.append(s)
        return ready

    def should_launch(self, ready: Sequence[Session], now: float) -> bool:
        """Start a tick now? At once when nothing is in flight; otherwise (below `depth`) once
        the oldest due frame has waited `coalesce_s`."""
        if not ready or len(self.ticks) >= self.depth:
            return False
        if not self.ticks:
            return True
        return now - min(s.next_due for s in ready) >= self.coalesce

    def launch(self, ready: Sequence[Session]) -> None:
        io, rel, px = [], [], 0
        for s in ready:
            rad, mot = self.rings[(s.width, s.height)]
            k = s.processed % rad.shape[0]
            io.append((s.stream.handle, rad[k], None, None, mot[k], s.out))
            rel.append((s.sid, s.next_due))
            px += s.width * s.height
            s.next_due += 1.0 / s.fps
            s.in_flight += 1
        start = torch.cuda.Event(enable_timing=True)
        start.record(self.cs)
        W.wrls_batch_tick(self.batch, io)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.cs)
        self.ticks.append(Tick(ev, rel, px, start))

    def poll(self, now: float) -> None:
        done = [t for t in self.ticks if t.event.query()]
        if not done:
            return
        t_done = time.perf_counter()
        for t in done:
            self.ticks.remove(t)
            self.pixels_done += t.pixels
            self.ticks_done += 1
            if t.start is not None:
                self.gpu_ms += t.start.elapsed_time(t.event)
            for sid, rel in t.releases:
                lat = t_done - rel
                self.latencies.append(lat)
                if lat > self.deadline:
                    self.missed += 1
                self.frames_done += 1
                s = self.active.get(sid)
                if s is not None:
                    s.in_flight -= 1
                    s.processed += 1
        for sid in [sid for sid, s in self.active.items() if s.in_flight == 0 and now >= s.depart]:
            self.depart(sid, now)

    def snapshot(self) -> Dict[int, Tuple[int, int, int, torch.Tensor]]:
        """Synchronise; {sid: (width, height, frames processed, copy of the last output)}."""
        self.cs.synchronize()
        self.poll(time.perf_counter())
        return {sid: (s.width, s.height, s.processed, s.out.clone()) for sid, s in self.active.items()}

    def close(self) -> None:
        self.cs.synchronize()
        for s in list(self.active.values()):
            s.stream.close()
        self.active.clear()
        self._evict(0)
        W.wrls_batch_destroy(self.batch)
        self.batch = 0


def make_rings(resolutions: Sequence[Tuple[int, int]], frames: int = 4, seed: int = 11,
               device="cuda") -> Dict[Tuple[int, int], Tuple[torch.Tensor, torch.Tensor]]:
    rings = {}
    for i, (w, h) in enumerate(resolutions):
        sc = synth.Scene(synth.SceneSpec(w, h, frames + 1, seed=seed + i, motion="orbit", firefly_frac=0.05))
        rad = torch.empty(frames, 3, h, w, device=device)
        mot = torch.empty(frames, 2, h, w, device=device)
        for t in range(frames):   # frames 1..K: frame 0 of a sequence has no motion
            f = sc.frame(t + 1, device=device)
            rad[t].copy_(f["radiance"])
            mot[t].copy_(f["motion"])
        rings[(w, h)] = (rad, mot)
    return rings


def calibrate_throughput(rings, params: Optional[W.wrls_params] = None, per_res: int = 2,
                         ticks: int = 20) -> float:
    """Pixels per second that batched ticks sustain on this GPU: `per_res` streams of every
    ring resolution in each tick, after a warm-up tick."""
    p = params if params is not None else W.wrls_params_default(state_precision=W.WRLS_STATE_BF16)
    cs = torch.cuda.Stream()
    b = W.wrls_batch_create(per_res * len(rings))
    W.wrls_batch_set_cuda_stream(b, cs)
    streams, io, px = [], [], 0
    for (w, h), (rad, mot) in rings.items():
        for _ in range(per_res):
            st = W.Stream(w, h, p, cuda_stream=cs)
            out = torch.empty(3, h, w, device="cuda")
            streams.append((st, out))
            io.append((st.handle, rad[0], None, None, mot[0], out))
            px += w * h
    W.wrls_batch_tick(b, io)
    cs.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record(cs)
    for _ in range(ticks):
        W.wrls_batch_tick(b, io)
    e.record(cs)
    e.synchronize()
    rate = px * ticks / (a.elapsed_time(e) / 1e3)
    W.wrls_batch_destroy(b)
    for st, _ in streams:
        st.close()
    return rate


def simulate(duration_s: float = 15.0, arrival_rate: float = 2.0, lifetime=(10.0, 60.0),
             resolutions=synth.SERVING_RESOLUTIONS, fps_range=(30.0, 60.0), max_sessions: int = 64,
             hbm_budget_bytes: Optional[int] = None, deadline_s: float = 1 / 60, depth: int = 2,
             seed: int = 5, warm_start: bool = True, params: Optional[W.wrls_params] = None,
             rings=None, rate_budget_mpix_s=None, rate_fraction: float = 0.9,
             coalesce_s: float = 0.0, capacity_px_s: Optional[float] = None) -> dict:
    """Run the serving loop in real time for `duration_s`. Sessions arrive as a Poisson
    process; with warm_start the run starts from the stationary population (Poisson count
    with mean arrival_rate * mean lifetime, residual lifetimes uniform), admitted before the
    clock starts (their streams are created then), each with its first frame due at a uniform
    random phase within its frame period after the start (a stationary population's sessions
    are not in phase).
    rate_budget_mpix_s: None = admission by memory and slots only; "auto" = rate_fraction x
    the throughput calibrate_throughput measures; a number = that budget in Mpix/s."""
    rng = random.Random(seed)
    if rings is None:
        rings = make_rings(resolutions)
    if hbm_budget_bytes is None:
        free, _ = torch.cuda.mem_get_info()
        hbm_budget_bytes = int(0.5 * free)
    capacity = capacity_px_s
    if rate_budget_mpix_s == "auto":
        if capacity is None:
            capacity = calibrate_throughput(rings, params)
        rate_budget_mpix_s = rate_fraction * capacity / 1e6
    srv = Server(hbm_budget_bytes, max_sessions=max_sessions, params=params, depth=depth,
                 deadline_s=deadline_s, rings=rings, coalesce_s=coalesce_s,
                 rate_budget_px_s=None if rate_budget_mpix_s is None else rate_budget_mpix_s * 1e6)
    t0 = time.perf_counter()
    sid = 0
    initial, residual = [], []
    if warm_start:
        mean_pop = arrival_rate * 0.5 * (lifetime[0] + lifetime[1])
        # Poisson(mean_pop) by inversion
        n, p, L = 0, 1.0, math.exp(-mean_pop)
        while True:
            p *= rng.random()
            if p <= L:
                break
            n += 1
        for _ in range(n):
            w, h = rng.choice(list(resolutions))
            life = rng.uniform(*lifetime)
            initial.append(Session(sid, w, h, rng.uniform(*fps_range), t0, math.inf))
            residual.append(rng.uniform(0, life))
            sid += 1
    for s in initial:
        srv.request(s, t0)
    t0 = time.perf_counter()     # the clock starts once the warm-start population is admitted
    phase = random.Random(seed + 7919)
    for s, r in zip(initial, residual):
        s.arrive, s.depart = t0, t0 + r
        if s.stream is not None:
            s.next_due = t0 + phase.uniform(0.0, 1.0 / s.fps)
    arrivals = []
    t = t0
    while True:
        t += rng.expovariate(arrival_rate)
        if t > t0 + duration_s:
            break
        w, h = rng.choice(list(resolutions))
        arrivals.append(Session(sid, w, h, rng.uniform(*fps_range), t, t + rng.uniform(*lifetime)))
        sid += 1
    pending = list(arrivals)
    end = t0 + duration_s
    rounds = 0
    with torch.cuda.stream(srv.cs):
        while True:
            now = time.perf_counter()
            if now >= end:
                break
            while pending and pending[0].arrive <= now:
                srv.request(pending.pop(0), now)
            for s in [s for s in srv.active.values() if now >= s.depart and s.in_flight == 0]:
                srv.depart(s.sid, now)
            srv.poll(now)
            if len(srv.ticks) < srv.depth:
                ready = srv.due_frames(now)
                if srv.should_launch(ready, now):
                    srv.launch(ready)
                    rounds += 1
        srv.cs.synchronize()
        srv.poll(time.perf_counter())
    wall = time.perf_counter() - t0
    lat = sorted(srv.latencies)

    def pct(q):
        return lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))] * 1e3 if lat else None
    res = {
        "duration_s": round(wall, 3), "frames": srv.frames_done, "ticks": rounds,
        "frames_per_tick": round(srv.frames_done / max(srv.ticks_done, 1), 2),
        "coalesce_ms": round(coalesce_s * 1e3, 3), "depth": depth,
        "mpix_per_s": round(srv.pixels_done / wall / 1e6, 2),
        "gpu_busy_fraction": round(srv.gpu_ms / 1e3 / wall, 4),
        "mpix_per_gpu_s": round(srv.pixels_done / max(srv.gpu_ms / 1e3, 1e-9) / 1e6, 1),
        "p50_ms": round(pct(0.50), 3) if lat else None, "p99_ms": round(pct(0.99), 3) if lat else None,
        "deadline_ms": round(deadline_s * 1e3, 2),
        "missed_or_dropped": srv.missed, "admitted": srv.admitted_total, "reused_streams": srv.reused,
        "max_concurrent": srv.max_concurrent, "queued_at_end": len(srv.queue),
        "hbm_budget_gb": round(hbm_budget_bytes / 1e9, 2), "hbm_used_gb_at_end": round(srv.used / 1e9, 3),
        "rate_budget_mpix_s": None if srv.rate_budget is None else round(srv.rate_budget / 1e6, 1),
        "calibrated_mpix_s": None if capacity is None else round(capacity / 1e6, 1),
        "admitted_rate_mpix_s_at_end": round(srv.rate / 1e6, 1),
    }
    srv.close()
    return res
