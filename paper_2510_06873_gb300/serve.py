"""Served form: a continuous-batching request loop over resident walkers.

Many metadynamics walkers (independent systems, each with its own hill
history) send requests "evaluate my next frame": positions in page-locked
host memory in, bias forces and CVs out.  The paper runs one walker per MD
process and hands its data over every step (Section "Frameworks of
GPU-MetaD"); this loop serves many such walkers from one GPU:

  * walker state (neighbour lists, hill history, grid, staging buffers) stays
    resident on the device between requests;
  * a request is admitted when its walker is idle and the walker's state
    fits the memory budget (idle walkers are evicted, least recently used,
    to make room: their hills go to host memory and come back on the next
    admission);
  * every admission point launches ONE batched step (metad_batch_step) over
    all admitted requests, so requests that arrive while others run on the
    GPU join the next launch, and up to `depth` launches are queued on the
    stream at once;
  * per-walker order is kept (one request of a walker in flight at a time),
    so each walker sees exactly the sequence of steps it would see alone;
    with the default tile a request's result is bit-identical alone and in
    the mix.

Latency is measured on the device clock: completion event minus the
request's arrival time, both relative to one start event.  The sequential
baseline (`run_plain`) serves the same trace one request at a time through
metad_step with a synchronisation after each.

All arithmetic runs in the library's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import metad as _m


@dataclass
class Request:
    walker: int
    index: int          # the walker's request number (0, 1, ...)
    arrival: float      # seconds after the start of the trace
    deposit: bool
    done: float = -1.0  # seconds after the start (device clock)
    cv: np.ndarray = None
    V: float = 0.0
    forces: np.ndarray = None
    err: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Walker:
    params: object               # metad_params
    centres: np.ndarray          # initial hill history [K, n_cv]
    heights: np.ndarray          # [K]
    frames: list                 # page-locked host tensors [n, 4]; request k uses frames[k % len]
    ctx: object = None           # Metad while resident
    pos_dev: torch.Tensor = None
    F_dev: torch.Tensor = None
    F_host: torch.Tensor = None  # page-locked [n, 3]
    bytes: int = 0
    busy: bool = False
    last_used: float = 0.0
    requests_done: int = 0
    evictions: int = 0
    saved: tuple = None          # (centres, heights) while evicted

    @property
    def n(self) -> int:
        return self.params.n_atoms


@dataclass
class ServeResult:
    requests: list
    makespan: float
    atom_steps: int
    batches: int
    mean_batch: float
    peak_bytes: int
    evictions: int
    launches: int = 0
    stats: dict = field(default_factory=dict)

    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.requests])
        return {"requests": len(self.requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "throughput_req_s": len(self.requests) / self.makespan,
                "atom_steps_per_s": self.atom_steps / self.makespan, "batches": self.batches,
                "mean_batch": self.mean_batch, "peak_device_bytes": self.peak_bytes, "evictions": self.evictions}


def walker_bytes(params) -> int:
    """Device bytes a resident walker holds: its context plus staging."""
    return _m.metad_estimate_bytes(params) + params.n_atoms * (16 + 12)


class Server:
    """Continuous-batching loop over `walkers` on `stream` (a torch stream
    whose handle every walker's params.stream already holds)."""

    def __init__(self, walkers, stream: torch.cuda.Stream, budget_bytes: int, deposit_every: int = 20,
                 depth: int = 2, keep_forces: bool = False, tile: int = 0):
        self.w = list(walkers)
        self.stream = stream
        self.dev = stream.device
        self.budget = int(budget_bytes)
        self.deposit_every = int(deposit_every)
        self.depth = max(1, int(depth))
        self.keep_forces = keep_forces
        self.tile = int(tile)
        for wk in self.w:
            wk.bytes = walker_bytes(wk.params)
            if wk.bytes > self.budget:
                raise ValueError(f"a walker needs {wk.bytes} bytes, more than the budget {self.budget}")
        self.resident = 0
        self.peak = 0
        self.batch = None
        self.batch_members = None  # walker ids of the batch object, in its order
        self.launches = 0          # batched steps
        self.kernel_launches = 0   # kernels of closed batch objects

    # ---------------------------------------------------------- residency
    def _make_resident(self, wid: int):
        wk = self.w[wid]
        with torch.cuda.stream(self.stream):
            wk.ctx = _m.Metad(wk.params)
            c, h = wk.saved if wk.saved is not None else (wk.centres, wk.heights)
            if len(h):
                wk.ctx.load_hills(c, h)
            wk.saved = None
            n = wk.n
            wk.pos_dev = torch.empty((n, 4), dtype=torch.float32, device=self.dev)
            wk.F_dev = torch.empty((n, 3), dtype=torch.float32, device=self.dev)
            if wk.F_host is None:
                wk.F_host = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        self.resident += wk.bytes
        self.peak = max(self.peak, self.resident)
        self._drop_batch()

    def _evict(self, wid: int):
        wk = self.w[wid]
        c, h = wk.ctx.get_hills()  # synchronises
        self._drop_batch()
        wk.saved = (c, h)
        wk.ctx.close()
        wk.ctx = None
        wk.pos_dev = wk.F_dev = None
        wk.evictions += 1
        self.resident -= wk.bytes

    def _drop_batch(self):
        if self.batch is not None:
            self.kernel_launches += self.batch.launch_count
            self.batch.close()  # synchronises its stream
            self.batch = None
            self.batch_members = None

    def _ensure_batch(self):
        if self.batch is None:
            ids = [k for k, wk in enumerate(self.w) if wk.ctx is not None]
            self.batch = _m.Batch([self.w[k].ctx for k in ids])
            if self.tile:
                self.batch.set_tile(self.tile)
            self.batch_members = ids
            self.slot_of = {wid: s for s, wid in enumerate(ids)}
            self.collect_bufs = [torch.zeros((len(ids), 4), dtype=torch.float64).pin_memory()
                                 for _ in range(self.depth + 1)]
            self.collect_next = 0

    def _admit(self, wid: int, now: float) -> bool:
        """Make walker wid resident if the budget allows (evicting idle
        walkers, least recently used first)."""
        wk = self.w[wid]
        if wk.ctx is not None:
            return True
        need = self.resident + wk.bytes - self.budget
        if need > 0:
            idle = sorted((w.last_used, k) for k, w in enumerate(self.w) if w.ctx is not None and not w.busy)
            freed, victims = 0, []
            for _, k in idle:
                if freed >= need:
                    break
                victims.append(k)
                freed += self.w[k].bytes
            if freed < need:
                return False
            for k in victims:
                self._evict(k)
        self._make_resident(wid)
        return True

    def preload(self) -> int:
        """Make walkers resident in order while the budget allows (before a
        trace, so that its requests find their state on the device)."""
        count = 0
        for k, wk in enumerate(self.w):
            if wk.ctx is None and self.resident + wk.bytes <= self.budget:
                self._make_resident(k)
                count += 1
        torch.cuda.synchronize(self.dev)
        return count

    # ---------------------------------------------------------- the loop
    def run(self, arrivals, walker_of) -> ServeResult:
        """Serve requests (arrival seconds, walker id) in real time."""
        reqs = []
        counts = collections.Counter()
        for t, wid in zip(arrivals, walker_of):
            k = counts[int(wid)]
            counts[int(wid)] += 1
            reqs.append(Request(int(wid), k, float(t), (k + 1) % self.deposit_every == 0))
        queue = collections.deque()
        inflight = collections.deque()
        nxt = 0
        batches, batch_sizes = 0, []
        with torch.cuda.stream(self.stream):
            start = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(self.dev)
            t0 = time.perf_counter()
            start.record(self.stream)
            while nxt < len(reqs) or queue or inflight:
                now = time.perf_counter() - t0
                while nxt < len(reqs) and reqs[nxt].arrival <= now:
                    queue.append(reqs[nxt])
                    nxt += 1
                while inflight and inflight[0][0].query():
                    self._retire(start, *inflight.popleft())
                if queue and len(inflight) < self.depth:
                    chosen = self._choose(queue, now)
                    if chosen:
                        inflight.append(self._launch(chosen))
                        batches += 1
                        batch_sizes.append(len(chosen))
                        continue
                if not inflight and not queue and nxt < len(reqs):
                    gap = reqs[nxt].arrival - (time.perf_counter() - t0)
                    if gap > 2e-3:
                        time.sleep(gap - 1e-3)  # idle GPU, nothing queued: wait for the next arrival
        done = [r for r in reqs]
        first = min(r.arrival for r in done)
        last = max(r.done for r in done)
        atom_steps = sum(self.w[r.walker].n for r in done)
        kernels = self.kernel_launches + (self.batch.launch_count if self.batch is not None else 0)
        return ServeResult(done, last - first, atom_steps, batches, float(np.mean(batch_sizes)) if batch_sizes else 0,
                           self.peak, sum(w.evictions for w in self.w), kernels)

    def _choose(self, queue, now):
        chosen, seen = [], set()
        keep = collections.deque()
        while queue:
            r = queue.popleft()
            wk = self.w[r.walker]
            if r.walker in seen or wk.busy or not self._admit(r.walker, now):
                seen.add(r.walker)  # later requests of this walker wait behind this one
                keep.append(r)
                continue
            seen.add(r.walker)
            wk.busy = True
            chosen.append(r)
        queue.extend(keep)
        return chosen

    def _launch(self, chosen):
        self._ensure_batch()
        m = len(self.batch_members)
        pos = [None] * m
        frc = [None] * m
        dep = np.zeros(m, dtype=np.int32)
        act = np.zeros(m, dtype=np.int32)
        for r in chosen:
            wk = self.w[r.walker]
            s = self.slot_of[r.walker]
            wk.pos_dev.copy_(wk.frames[r.index % len(wk.frames)], non_blocking=True)
            pos[s], frc[s] = wk.pos_dev, wk.F_dev
            dep[s] = 1 if r.deposit else 0
            act[s] = 1
        self.batch.step(pos, frc, accumulate=False, deposit=dep, active=act)
        for r in chosen:
            wk = self.w[r.walker]
            wk.F_host.copy_(wk.F_dev, non_blocking=True)
        buf = self.collect_bufs[self.collect_next]
        self.collect_next = (self.collect_next + 1) % len(self.collect_bufs)
        self.batch.collect(buf.numpy())
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        self.launches += 1
        return ev, chosen, buf, dict(self.slot_of)

    def _retire(self, start, ev, chosen, buf, slot_of):
        t = start.elapsed_time(ev) / 1e3
        out = buf.numpy()
        for r in chosen:
            wk = self.w[r.walker]
            s = slot_of[r.walker]
            r.done = t
            r.cv = out[s, :2].copy()
            r.V = float(out[s, 2])
            r.err = int(out[s, 3])
            if self.keep_forces:
                r.forces = wk.F_host.numpy().copy()
            wk.busy = False
            wk.last_used = t
            wk.requests_done += 1

    def close(self):
        self._drop_batch()
        for wk in self.w:
            if wk.ctx is not None:
                wk.ctx.close()
                wk.ctx = None


def run_plain(walkers, stream: torch.cuda.Stream, arrivals, walker_of, deposit_every: int = 20,
              keep_forces: bool = False) -> ServeResult:
    """Sequential plain evaluation of the same trace: one request at a time,
    metad_step on the walker's own context, synchronised after each."""
    dev = stream.device
    reqs = []
    counts = collections.Counter()
    for t, wid in zip(arrivals, walker_of):
        k = counts[int(wid)]
        counts[int(wid)] += 1
        reqs.append(Request(int(wid), k, float(t), (k + 1) % deposit_every == 0))
    with torch.cuda.stream(stream):
        for wk in walkers:
            if wk.ctx is None:
                wk.ctx = _m.Metad(wk.params)
                if len(wk.heights):
                    wk.ctx.load_hills(wk.centres, wk.heights)
                wk.pos_dev = torch.empty((wk.n, 4), dtype=torch.float32, device=dev)
                wk.F_dev = torch.empty((wk.n, 3), dtype=torch.float32, device=dev)
                if wk.F_host is None:
                    wk.F_host = torch.empty((wk.n, 3), dtype=torch.float32).pin_memory()
        start = torch.cuda.Event(enable_timing=True)
        ev = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        start.record(stream)
        for r in reqs:
            while time.perf_counter() - t0 < r.arrival:
                pass
            wk = walkers[r.walker]
            wk.pos_dev.copy_(wk.frames[r.index % len(wk.frames)], non_blocking=True)
            wk.ctx.step(wk.pos_dev, wk.F_dev, deposit=r.deposit)
            wk.F_host.copy_(wk.F_dev, non_blocking=True)
            ev.record(stream)
            cv, V, _ = wk.ctx.read_results()  # synchronises
            r.done = start.elapsed_time(ev) / 1e3
            r.cv = np.array([cv[0], cv[1] if len(cv) > 1 else 0.0])
            r.V = V
            if keep_forces:
                r.forces = wk.F_host.numpy().copy()
    first = min(r.arrival for r in reqs)
    last = max(r.done for r in reqs)
    atom_steps = sum(walkers[r.walker].n for r in reqs)
    return ServeResult(reqs, last - first, atom_steps, len(reqs), 1.0, 0, 0)
