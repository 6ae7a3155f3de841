"""Continuously batching request server for HEALPix transforms on one GPU.

Requests (map2alm or alm2map of 1..max_channels channels at some Nside) are
queued per (nside, lmax, op).  Whenever a slot -- a plan with its own CUDA
stream and I/O buffers, resident on the device -- is free, the oldest queue
with a slot of its geometry packs as many of its waiting requests as fit
into one batched call (hpx_map2alm_n / hpx_alm2map_n) of up to the slot's
batch capacity, which the executor sets per geometry and which may exceed
one request's channel limit, so that one pass over the Legendre functions
serves several requests: requests that arrive
while others run join the next batch, and slots of different geometries run
concurrently on their own streams.  New slots are admitted only while the
device bytes of all resident slots stay under the HBM cap; idle slots of
other geometries are evicted (least recently used) to make room.  Invalid
requests are completed at once with an error and never block the others.

The scheduling logic is plain Python over an executor interface, so it is
tested on the CPU with a fake executor; GpuExecutor runs it on libhpx.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

MAX_NSIDE = 2048


@dataclasses.dataclass
class Request:
    rid: int
    op: str                 # "map2alm" or "alm2map"
    nside: int
    nch: int
    x: object = None        # input: [nch, npix] real or [nch, nalm] complex
    t_arrival: float = 0.0  # seconds on the server clock
    lmax: int | None = None
    t_start: float | None = None
    t_done: float | None = None
    y: object = None
    error: str | None = None

    def __post_init__(self):
        if self.lmax is None:
            self.lmax = 3 * self.nside - 1

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrival


@dataclasses.dataclass
class Slot:
    key: tuple              # (nside, lmax)
    nbytes: int
    handle: object          # executor-specific
    busy: bool = False
    batch: list = dataclasses.field(default_factory=list)
    last_used: float = 0.0


class Server:
    def __init__(self, executor, hbm_cap_bytes: float = 120e9, max_channels: int = 32,
                 max_slots_per_key: int = 2, clock=time.perf_counter):
        self.ex = executor
        self.cap = hbm_cap_bytes
        self.max_ch = max_channels
        self.max_slots = max_slots_per_key
        self.clock = clock
        self.queues: dict = collections.OrderedDict()
        self.slots: dict = collections.defaultdict(list)
        self.bytes = 0
        self.peak_bytes = 0
        self.batches = 0
        self.evictions = 0
        self.known_bytes: dict = {}  # measured device bytes of a built slot, by geometry
        self.builds: collections.Counter = collections.Counter()  # slots built, by geometry
        self.finished: list = []

    def capacity(self, nside: int, lmax: int) -> int:
        """Channels one batch of this geometry may hold (the executor's
        choice, else the per-request limit)."""
        f = getattr(self.ex, "batch_capacity", None)
        return max(self.max_ch, int(f(nside, lmax))) if f else self.max_ch

    # -- admission ------------------------------------------------------------
    def submit(self, req: Request) -> None:
        err = None
        if req.op not in ("map2alm", "alm2map"):
            err = f"unknown op {req.op!r}"
        elif not (1 <= req.nside <= MAX_NSIDE and req.nside & (req.nside - 1) == 0):
            err = f"nside {req.nside} is not a power of two in [1, {MAX_NSIDE}]"
        elif not (1 <= req.nch <= self.max_ch):
            err = f"{req.nch} channels outside [1, {self.max_ch}]"
        elif req.lmax < 0:
            err = f"lmax {req.lmax} < 0"
        elif self.ex.slot_bytes(req.nside, req.lmax, self.capacity(req.nside, req.lmax)) > self.cap:
            err = "one slot for this request exceeds the HBM cap"
        if err is not None:
            req.error = err
            req.t_done = req.t_start = self.clock()
            self.finished.append(req)
            return
        self.queues.setdefault((req.nside, req.lmax, req.op), collections.deque()).append(req)

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def busy(self) -> bool:
        return any(s.busy for ss in self.slots.values() for s in ss)

    # -- slots ------------------------------------------------------------------
    def _free_slot(self, key, now):
        for s in self.slots[key]:
            if not s.busy:
                return s
        if len(self.slots[key]) >= self.max_slots:
            return None
        cap_ch = self.capacity(key[0], key[1])
        # the executor's estimate is an upper bound (it cannot know which
        # Legendre values are significant); once a slot of this geometry has
        # been built, its measured size is used instead
        need = self.known_bytes.get(key) or self.ex.slot_bytes(key[0], key[1], cap_ch)
        while self.bytes + need > self.cap:  # evict idle slots of other geometries, least recently used first
            idle = [s for k, ss in self.slots.items() if k != key for s in ss if not s.busy]
            if not idle:
                return None
            victim = min(idle, key=lambda s: s.last_used)
            self.slots[victim.key].remove(victim)
            self.ex.free_slot(victim.handle)
            self.bytes -= victim.nbytes
            self.evictions += 1
        handle = self.ex.new_slot(key[0], key[1], cap_ch)
        s = Slot(key=key, nbytes=self.ex.handle_bytes(handle), handle=handle, last_used=now)
        self.known_bytes[key] = s.nbytes
        self.builds[key] += 1
        self.slots[key].append(s)
        self.bytes += s.nbytes
        self.peak_bytes = max(self.peak_bytes, self.bytes)
        return s

    # -- one scheduling pass ------------------------------------------------------
    def pump(self) -> list:
        now = self.clock()
        done = []
        for ss in self.slots.values():
            for s in ss:
                if s.busy and self.ex.done(s.handle):
                    ys = self.ex.finish(s.handle)
                    t = self.clock()
                    for r, y in zip(s.batch, ys):
                        r.y, r.t_done = y, t
                        done.append(r)
                    s.busy, s.batch, s.last_used = False, [], t
        # oldest waiting request first
        order = sorted((q[0].t_arrival, k) for k, q in self.queues.items() if q)
        for _, k in order:
            q = self.queues[k]
            while q:
                s = self._free_slot((k[0], k[1]), now)
                if s is None:
                    break
                batch, nch = [], 0
                cap_ch = self.capacity(k[0], k[1])
                while q and nch + q[0].nch <= cap_ch:
                    r = q.popleft()
                    r.t_start = now
                    batch.append(r)
                    nch += r.nch
                s.busy, s.batch = True, batch
                self.ex.launch(s.handle, k[2], batch)
                self.batches += 1
        self.finished.extend(done)
        return done

    def run(self, requests, t0: float | None = None, drain_s: float = 30.0, idle_sleep: float = 2e-4):
        """Feed requests (sorted by t_arrival, seconds from t0) as their
        arrival times pass, until all are done or drain_s after the last
        arrival.  Returns the wall time used."""
        t0 = self.clock() if t0 is None else t0
        i, n = 0, len(requests)
        t_last = requests[-1].t_arrival if n else 0.0
        while True:
            now = self.clock() - t0
            while i < n and requests[i].t_arrival <= now:
                requests[i].t_arrival += t0  # to the server clock
                self.submit(requests[i])
                i += 1
            self.pump()
            if i == n and not self.pending() and not self.busy():
                break
            if now > t_last + drain_s:
                break
            if i < n and not self.busy() and not self.pending():
                time.sleep(min(idle_sleep, max(0.0, requests[i].t_arrival - now)))
            else:  # a batch is running: poll again at once (a short sleep oversleeps by tens of us)
                time.sleep(0)
        return self.clock() - t0


def latency_report(requests) -> dict:
    lat = np.array([r.latency for r in requests if r.t_done is not None and r.error is None])
    served = len(lat)
    out = {"requests": len(requests), "served": served,
           "errors": sum(1 for r in requests if r.error is not None)}
    if served:
        out.update({"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "mean_ms": float(lat.mean() * 1e3)})
    return out


# ----------------------------------------------------------------------------
# libhpx executor
# ----------------------------------------------------------------------------
class GpuExecutor:
    """Slots are libhpx plans (FP32) with a CUDA stream and one map and one
    coefficient buffer of the slot's batch capacity.

    table_nsides: geometries whose slots hold a plan-time lambda table on the
    tensor cores (FP16 hi/lo split products, FP32 accuracy); streamed_nsides:
    geometries whose slots recompute lambda per call into streamed blocks
    contracted on the tensor cores (no table held; one recurrence per
    batch whatever its channel count); the others recompute lambda on the
    CUDA cores, once per group of channels of a launch.
    batch_channels: channels per batch by Nside (default 32); one batch runs
    the recurrence, or streams the table, once for all its requests."""

    def __init__(self, device=None, keep_outputs: bool = True, lambda_table_nsides=(), batch_channels=None,
                 tensor_cores: bool = True, streamed_nsides=()):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.keep = keep_outputs
        self.table_nsides = set(lambda_table_nsides)
        self.streamed_nsides = set(streamed_nsides) - self.table_nsides
        self.batch_channels = dict(batch_channels or {})
        self.tc = tensor_cores

    def batch_capacity(self, nside, lmax) -> int:
        return int(self.batch_channels.get(nside, 32))

    def _flags(self, nside) -> int:
        from . import _lib
        if nside in self.streamed_nsides:
            return _lib.HPX_PLAN_LAMBDA_TABLE | _lib.HPX_PLAN_TENSOR_CORES | _lib.HPX_PLAN_LAMBDA_STREAM
        if nside not in self.table_nsides:
            return _lib.HPX_PLAN_LAMBDA_RECOMPUTE
        return _lib.HPX_PLAN_LAMBDA_TABLE | (_lib.HPX_PLAN_TENSOR_CORES if self.tc else 0)

    def slot_bytes(self, nside, lmax, max_ch) -> int:
        from . import _lib
        plan = _lib.lib().hpx_plan_estimate_bytes(nside, lmax, lmax, max_ch, _lib.HPX_F32, self._flags(nside))
        io = max_ch * (4 * 12 * nside * nside + 8 * ((lmax + 1) * (lmax + 2) // 2))
        return int(plan + io)

    def new_slot(self, nside, lmax, max_ch):
        from . import Plan
        torch = self.torch
        tab = nside in self.table_nsides
        if nside in self.streamed_nsides:
            plan = Plan(nside, lmax, lmax, max_ch, "f32", streamed=True, device=self.device)
        else:
            plan = Plan(nside, lmax, lmax, max_ch, "f32", lambda_table=tab, tensor_cores=tab and self.tc,
                        device=self.device)
        h = {"plan": plan, "stream": torch.cuda.Stream(self.device), "map": plan.empty_map(),
             "alm": plan.empty_alm(), "event": torch.cuda.Event(), "ys": []}
        h["nbytes"] = plan.device_bytes + h["map"].nbytes + h["alm"].nbytes
        return h

    def handle_bytes(self, h) -> int:
        return int(h["nbytes"])

    def free_slot(self, h) -> None:
        h["stream"].synchronize()
        h["plan"].close()
        h.clear()

    def launch(self, h, op, batch) -> None:
        torch = self.torch
        plan, st = h["plan"], h["stream"]
        src, dst = (h["map"], h["alm"]) if op == "map2alm" else (h["alm"], h["map"])
        with torch.cuda.stream(st):
            off = 0
            for r in batch:
                src[off: off + r.nch].copy_(r.x, non_blocking=True)
                off += r.nch
            if op == "map2alm":
                plan.map2alm_n(off, src, dst, stream=st)
            else:
                plan.alm2map_n(off, src, dst, stream=st)
            ys, off = [], 0
            for r in batch:
                ys.append(dst[off: off + r.nch].clone() if self.keep else None)
                off += r.nch
            h["event"].record(st)
        h["ys"] = ys

    def done(self, h) -> bool:
        return h["event"].query()

    def finish(self, h):
        ys, h["ys"] = h["ys"], []
        return ys


def make_requests(seed: int, rate: float, duration: float, nside_weights: dict, max_channels: int = 32,
                  op_mix: float = 0.5):
    """Seeded Poisson arrivals; op map2alm with probability op_mix; Nside
    drawn from nside_weights; channels uniform in 1..max_channels."""
    from . import synthetic as syn
    t = syn.poisson_arrivals(seed, rate, duration)
    g = syn.rng(seed + 1)
    ns = np.array(sorted(nside_weights))
    w = np.array([nside_weights[k] for k in ns], np.float64)
    pick = g.choice(len(ns), size=len(t), p=w / w.sum())
    ops = g.uniform(size=len(t)) < op_mix
    nch = g.integers(1, max_channels + 1, size=len(t))
    return [Request(rid=i, op="map2alm" if ops[i] else "alm2map", nside=int(ns[pick[i]]), nch=int(nch[i]),
                    t_arrival=float(t[i])) for i in range(len(t))]
