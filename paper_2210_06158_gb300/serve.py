"""Serving loop for many render sessions: admission by a device-memory budget and
continuous batching of frame requests over dof_batch_frame.

Requests (a session wants its next frame) arrive at any time.  Each tick the server
  * retires finished batches (latency = completion - arrival),
  * starts a new batch from the pending requests as soon as fewer than `max_inflight`
    batches are on the GPU: at most one request per session (its history is
    sequential) and at most `max_batch` requests, oldest first,
so requests that arrive while others are on the GPU join the next batch and their
work overlaps the running one (two streams).  A session whose newer request arrives
before the older one started keeps only the newest (a real-time renderer shows the
latest camera); the superseded request is counted as dropped.

The executor does the work; GpuExecutor drives the CUDA library, FakeExecutor models
the cost on a virtual clock (host-only tests of the scheduling logic).
"""

from __future__ import annotations

import collections
import gc
import math
import time
from dataclasses import dataclass, field


@dataclass
class SessionSpec:
    name: str
    width: int
    height: int
    fps: float                     # arrival rate of frame requests
    scene: object = None           # synth.Scene
    params: dict = field(default_factory=dict)
    poses: list = field(default_factory=list)   # camera poses cycled by frame index
    intr: dict = field(default_factory=dict)


@dataclass
class Request:
    session: int
    arrival: float
    frame: int
    start: float = -1.0
    done: float = -1.0


def percentile(xs, q):
    if not xs:
        return float("nan")
    s = sorted(xs)
    k = min(len(s) - 1, max(0, int(math.ceil(q / 100.0 * len(s))) - 1))
    return s[k]


# ---------------------------------------------------------------------------
# executors
# ---------------------------------------------------------------------------

class FakeExecutor:
    """Virtual-clock executor: a batch takes fixed_ms + sum of per-pixel costs."""

    def __init__(self, budget_bytes, ms_per_mpix=0.5, fixed_ms=0.05, bytes_per_px=400, fail_on=None):
        self.budget = budget_bytes
        self.used = 0
        self.ms_per_mpix, self.fixed_ms, self.bytes_per_px = ms_per_mpix, fixed_ms, bytes_per_px
        self.now = 0.0
        self.gpu_free_at = [0.0, 0.0]
        self.sessions = {}
        self.fail_on = fail_on or set()
        self._next = 0

    def clock(self):
        return self.now

    def advance(self, t):
        self.now = max(self.now, t)

    def estimate_bytes(self, spec):
        return spec.width * spec.height * self.bytes_per_px

    def open(self, sid, spec):
        b = self.estimate_bytes(spec)
        if self.used + b > self.budget:
            raise MemoryError("budget")
        self.used += b
        self.sessions[sid] = (spec, b)

    def close(self, sid):
        spec, b = self.sessions.pop(sid)
        self.used -= b

    def submit(self, reqs, stream):
        if any(r.session in self.fail_on for r in reqs):
            raise RuntimeError("executor failure")
        cost = self.fixed_ms + sum(self.sessions[r.session][0].width * self.sessions[r.session][0].height
                                   for r in reqs) / 1e6 * self.ms_per_mpix
        start = max(self.now, self.gpu_free_at[stream])
        end = start + cost / 1e3
        self.gpu_free_at[stream] = end
        self._next += 1
        return (self._next, end)

    def done(self, token):
        return self.now >= token[1]

    def finish_time(self, token):
        return token[1]

    def next_event(self):
        return min(self.gpu_free_at)


class GpuExecutor:
    """Drives libdof: per admitted session a device scene (BVH), a history and a small
    ring of device G-buffers rendered by the G-buffer producer; batches go through
    dof_batch_frame on one of two streams, completion is an event.  per_frame: each
    request of a batch runs as its own dof_frame instead (the plain per-frame form);
    fp16: the sessions store their colour image buffers in FP16 (FP32 arithmetic).
    record: every served frame's image is copied (on its stream, after its batch) into
    `records[(session, frame)]`, so that each can be compared with the same frame
    rendered alone."""

    def __init__(self, budget_bytes, device=0, gbuf_ring=2, per_frame=False, fp16=False, record=False):
        import torch
        from . import dof
        self.torch, self.dof = torch, dof
        self.per_frame, self.fp16 = per_frame, fp16
        self.gathers = {}              # image storage (fp16) -> the gathers' tuned settings
        self.record = record
        self.records = {}
        self.ctx = dof.Context(device, mem_budget_bytes=budget_bytes)
        self.ctx.set_trace(stats=False)    # served frames need no node-visit counters
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(2)]
        self.sessions = {}
        self.ring = gbuf_ring
        self.t0 = time.perf_counter()

    def clock(self):
        return time.perf_counter() - self.t0

    def advance(self, t):
        dt = t - self.clock()
        if dt > 0:
            time.sleep(min(dt, 0.0005))

    def estimate_bytes(self, spec):
        hpx = (spec.width // 2) * (spec.height // 2)
        mr = int(spec.params.get("spp", 1)) if int(spec.params.get("ray_mode", 0)) == 0 else int(spec.params.get("m", 1))
        return int(hpx * (411 + 36 * mr) + spec.scene.n_tris * 112)

    def open(self, sid, spec):
        from synth.scenes import Camera
        dof, torch = self.dof, self.torch
        try:
            scene = dof.Scene(self.ctx, spec.scene)
            mr = int(spec.params.get("spp", 1)) if int(spec.params.get("ray_mode", 0)) == 0 else int(spec.params.get("m", 1))
            hist = dof.History(self.ctx, spec.width, spec.height, max_rays=mr)
        except dof.DofError as e:
            if e.code in (-2, -3):
                raise MemoryError(str(e))
            raise
        gbs = []
        for k in range(self.ring):
            cam = Camera.from_poses(spec.intr, spec.poses[k % len(spec.poses)])
            g = dof.gbuffer(self.ctx, scene, cam, spec.params, spec.width, spec.height)
            del g["prim"]
            gbs.append(g)
        out = torch.empty((spec.height, spec.width, 4), dtype=torch.float32, device=self.device)
        prm = dict(spec.params, image_storage=1) if self.fp16 else spec.params
        self.sessions[sid] = dict(spec=spec, scene=scene, hist=hist, gbs=gbs, out=out,
                                  pstruct=dof.params_struct(prm))
        torch.cuda.synchronize()

    def tune(self, frames=2, max_batch=32):
        """Autotune the tracer (tune.tune_trace) and then the gathers' launch settings
        (tune.tune_gathers, once per image storage: FP16 texels are smaller) on batched
        steps of the admitted sessions (up to max_batch of them, one frame each), as a
        server does at start-up.  The context keeps the tracer's pick and the gathers'
        pick of the current form (set_form applies the pick of its storage); every
        history starts afresh.  Returns the tracer's pick."""
        from . import tune
        sids = list(self.sessions)[:max_batch]
        st = self.streams[0]

        def step(k):
            items = []
            for sid in sids:
                s = self.sessions[sid]
                items.append(dict(scene=s["scene"], gbuf=s["gbs"][k % self.ring], cam=self.camera(s, k),
                                  params=s["pstruct"], hist=s["hist"], out=s["out"]))
            self.dof.batch_frame(self.ctx, items, stream=st)

        best, _ = tune.tune_trace(self.ctx, step, frames=frames, stream=st)
        fp16 = self.fp16
        for f16 in (not fp16, fp16):
            self.set_form(self.per_frame, f16)
            self.gathers[f16], _ = tune.tune_gathers(self.ctx, step, frames=frames, stream=st)
        self.set_form(self.per_frame, fp16)
        return best

    def set_form(self, per_frame=False, fp16=False):
        """Switch every admitted session to the given form (batched or per-frame, FP16 or
        FP32 image storage) and start its history afresh."""
        self.torch.cuda.synchronize()
        self.per_frame, self.fp16 = per_frame, fp16
        g = self.gathers.get(fp16)
        if g is not None:
            self.ctx.set_gather(block=g["gather_block"], main_form=g["main_form"], recon_block=g["recon_block"])
        for s in self.sessions.values():
            prm = dict(s["spec"].params, image_storage=1) if fp16 else s["spec"].params
            s["pstruct"] = self.dof.params_struct(prm)
            s["hist"].reset()

    def close(self, sid):
        s = self.sessions.pop(sid)
        s["hist"].close()
        s["scene"].close()

    def camera(self, s, frame):
        """Camera of frame `frame`: the pose of its G-buffer (the ring cycles the first
        `gbuf_ring` poses) and the previous frame's pose."""
        from synth.scenes import Camera
        spec = s["spec"]
        n = min(self.ring, len(spec.poses))
        cam = Camera.from_poses(spec.intr, spec.poses[frame % n], spec.poses[(frame - 1) % n] if frame else None,
                                frame_index=frame)
        return self.dof.camera_struct(cam)

    def submit(self, reqs, stream):
        items = []
        for r in reqs:
            s = self.sessions[r.session]
            items.append(dict(scene=s["scene"], gbuf=s["gbs"][r.frame % self.ring], cam=self.camera(s, r.frame),
                              params=s["pstruct"], hist=s["hist"], out=s["out"]))
        st = self.streams[stream]
        if self.per_frame:
            for it in items:
                self.dof.frame(self.ctx, it["scene"], it["gbuf"], None, None, it["hist"], it["out"], stream=st,
                               cam_struct=it["cam"], params_s=it["params"])
        else:
            self.dof.batch_frame(self.ctx, items, stream=st)
        if self.record:
            with self.torch.cuda.stream(st):
                for r, it in zip(reqs, items):
                    self.records[(r.session, r.frame)] = it["out"].clone()
        ev = self.torch.cuda.Event()
        ev.record(st)
        return ev

    def done(self, token):
        return token.query()

    def finish_time(self, token):
        return self.clock()

    def next_event(self):
        return self.clock() + 0.0002


# ---------------------------------------------------------------------------
# server
# ---------------------------------------------------------------------------

class Server:
    def __init__(self, executor, max_batch=32, max_inflight=2):
        self.ex = executor
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.specs = {}
        self.rejected = []

    def admit(self, sid, spec) -> bool:
        """Admit a session if its scene, history and buffers fit the budget."""
        try:
            self.ex.open(sid, spec)
        except MemoryError:
            self.rejected.append(sid)
            return False
        self.specs[sid] = spec
        return True

    def release(self, sid):
        self.ex.close(sid)
        self.specs.pop(sid, None)

    def run(self, arrivals):
        """Serve `arrivals` (list of (time_s, session id), sorted by time, times relative
        to the start of the run) to completion.  Returns the statistics: frames, dropped,
        failed, p50/p99 latency (ms), frames/s, and per-session completed frame numbers."""
        # no cyclic garbage collection while serving: a full pass over the process's
        # objects can hold the loop for tens of milliseconds and lands in the tail latency
        gc_was_on = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            return self._run(arrivals)
        finally:
            if gc_was_on:
                gc.enable()

    def _run(self, arrivals):
        base = self.ex.clock()
        arrivals = collections.deque((t + base, sid) for t, sid in arrivals if sid in self.specs)
        pending = collections.OrderedDict()     # session -> Request (newest only)
        busy = set()                            # sessions with a frame on the GPU
        inflight = []                           # (token, [requests], stream)
        frame_no = collections.Counter()
        done, dropped, failed = [], 0, []
        batches = []
        stream_busy = [False] * self.max_inflight
        t_first = arrivals[0][0] if arrivals else base
        while arrivals or pending or inflight:
            now = self.ex.clock()
            while arrivals and arrivals[0][0] <= now:
                t, sid = arrivals.popleft()
                if sid not in self.specs:
                    continue                    # evicted
                if sid in pending:
                    dropped += 1
                    pending.pop(sid)
                pending[sid] = Request(sid, t, frame_no[sid])
                frame_no[sid] += 1
            still = []
            for tok, reqs, st in inflight:
                if self.ex.done(tok):
                    tf = self.ex.finish_time(tok)
                    for r in reqs:
                        r.done = tf
                        busy.discard(r.session)
                        done.append(r)
                    stream_busy[st] = False
                else:
                    still.append((tok, reqs, st))
            inflight = still
            launched = False
            if pending and len(inflight) < self.max_inflight:
                batch = [r for sid, r in pending.items() if sid not in busy][: self.max_batch]
                if batch:
                    st = stream_busy.index(False)
                    for r in batch:
                        pending.pop(r.session)
                        r.start = now
                    try:
                        tok = self.ex.submit(batch, st)
                    except Exception:
                        # the batch failed as a whole: its sessions are evicted, the others go on
                        for r in batch:
                            failed.append(r)
                            if r.session in self.specs:
                                self.release(r.session)
                        continue
                    for r in batch:
                        busy.add(r.session)
                    stream_busy[st] = True
                    inflight.append((tok, batch, st))
                    batches.append(len(batch))
                    launched = True
            if not launched:
                nxt = [arrivals[0][0]] if arrivals else []
                if inflight:
                    nxt.append(min(self.ex.finish_time(t) if isinstance(self.ex, FakeExecutor) else now + 2e-4
                                   for t, _, _ in inflight))
                if nxt:
                    self.ex.advance(min(nxt))
        lat = [(r.done - r.arrival) * 1e3 for r in done]
        t_last = max((r.done for r in done), default=t_first)
        span = max(t_last - t_first, 1e-9)
        per_session = collections.defaultdict(list)
        for r in sorted(done, key=lambda r: r.done):
            per_session[r.session].append(r.frame)
        return dict(frames=len(done), dropped=dropped, failed=len(failed), p50_ms=percentile(lat, 50),
                    p99_ms=percentile(lat, 99), mean_ms=sum(lat) / len(lat) if lat else float("nan"),
                    frames_per_s=len(done) / span, admitted=len(self.specs), rejected=len(self.rejected),
                    mean_batch=sum(batches) / len(batches) if batches else 0.0, max_batch=max(batches, default=0),
                    per_session=dict(per_session))


def poisson_arrivals(rng_seed, sessions, duration_s):
    """Seeded Poisson arrivals: per session exponential gaps at its fps."""
    import numpy as np
    rng = np.random.default_rng(rng_seed)
    out = []
    for sid, spec in sessions.items():
        t = float(rng.exponential(1.0 / spec.fps))
        while t < duration_s:
            out.append((t, sid))
            t += float(rng.exponential(1.0 / spec.fps))
    out.sort()
    return out
