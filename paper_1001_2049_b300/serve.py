"""Continuous-batching render server over resident cubes.

The paper's thin client turns user interaction into render commands for the
scheduler (Fig. 1 caption) and its framework aims at interactive control of
the rendering (abstract; §3.1 module 4).  This module is that loop on one
GPU: render requests (a camera, a resolution, a mode and a transfer
function for one of the resident cubes) arrive at any time; the server

  * admits a request when a launch slot is free and its output image fits in
    the memory budget still unused by requests in flight (admission by
    memory, first come first served);
  * batches admitted work into one persistent launch (``vr_render_batch``)
    on the next free stream, so requests that arrive while others are on the
    GPU run in the next launch, overlapping the running one on the device
    (continuous batching).  A launch takes at most ``launch_rays`` rays, and
    an image larger than ``band_rays`` is split into row bands (the same rays
    bit for bit, each band a request of its own), so one large view cannot
    hold a launch -- and the requests arriving behind it -- for long;
  * sees each request finish individually through its completion word in
    page-locked host memory, written by the kernel once the request's image
    is complete, and records its latency (completion - arrival, host
    monotonic clock) for p50 / p99;
  * can cancel a request: not yet admitted, it is dropped; admitted, its
    bands not yet launched are dropped and the rest run out (a launched
    kernel is not interrupted), and it is reported as cancelled.

All rendering is done by the library's kernels; this is host-side control.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .api import MODES, Request, Volume, batch_workspace, render_batch
from ._lib import VR_COMPOSITE


def plan_bands(h: int, w: int, band_rays: int):
    """Row bands (row0, rows) covering an h x w image, each of about
    ``band_rays`` rays (whole rows; 0 or an image within the limit: one band
    of every row)."""
    if band_rays <= 0 or h * w <= band_rays:
        return [(0, h)]
    rows = max(1, band_rays // max(1, w))
    return [(r, min(rows, h - r)) for r in range(0, h, rows)]


def take_units(queue, max_units: int, launch_rays: int):
    """Pop the units of the next launch from the front of ``queue`` (first
    come, first served): at most ``max_units`` and, beyond the first, no
    more than ``launch_rays`` rays in all (0: no ray limit)."""
    out, rays = [], 0
    while queue and len(out) < max_units:
        u = queue[0]
        if out and launch_rays > 0 and rays + u.rays > launch_rays:
            break
        out.append(queue.popleft())
        rays += u.rays
    return out


@dataclass
class RenderJob:
    """One render request as submitted to the server."""
    cube: str
    cam: np.void
    w: int
    h: int
    mode: str = "composite"
    step: float = 0.5
    tf: tuple | None = None
    arrival: float = 0.0                 # host monotonic time, set on submit
    admitted: float = 0.0
    finished: float = 0.0
    out: torch.Tensor | None = None
    ticket: int = -1
    cancelled: bool = False
    units: int = 0                       # bands to render (planned, less any cancelled)
    launched: int = 0                    # bands handed to a launch
    seen: int = 0                        # bands seen complete (done word or launch)
    retired: int = 0                     # bands whose launch has completed

    @property
    def out_bytes(self):
        return self.w * self.h * (16 if MODES[self.mode] == VR_COMPOSITE else 4)

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class _Unit:
    """One row band of a job: one request of a batched launch."""
    job: RenderJob
    row0: int
    rows: int
    seen: bool = False

    @property
    def rays(self):
        return self.rows * self.job.w


@dataclass
class _Launch:
    units: list
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    flags: torch.Tensor | None          # pinned int32, one per unit (batched launches)
    issued: float = 0.0


class Server:
    """Render server over ``volumes`` (name -> Volume, resident on the GPU).

    ``mem_budget`` bounds the bytes of output images of requests in flight;
    ``max_batch`` the requests (bands) per launch; ``streams`` the launches
    that can be on the device at once; ``band_rays`` the rays of a row band
    (0: images are not split) and ``launch_rays`` the rays of a launch (0: no
    limit).  ``per_request`` renders each request with its own single-view
    render call (``Volume.render``) instead of batched launches: the plain
    path the batched one is compared with.
    ``resident`` holds, per cube, the device bytes it keeps for the whole
    run (library-owned texture storage and MIP bounds, caller-owned bricks
    and masks), which the output budget comes on top of.
    """

    def __init__(self, volumes: dict, mem_budget: int = 1 << 30, max_batch: int = 64,
                 streams: int = 2, keep_outputs: bool = False, per_request: bool = False,
                 band_rays: int = 0, launch_rays: int = 0):
        self.volumes = volumes
        self.per_request = per_request
        self.mem_budget = int(mem_budget)
        self.max_batch = int(max_batch)
        self.keep_outputs = keep_outputs
        self.band_rays = 0 if per_request else int(band_rays)
        self.launch_rays = 0 if per_request else int(launch_rays)
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.workspaces = [batch_workspace() for _ in range(streams)]
        self.free_streams = collections.deque(range(streams))
        self.pending = collections.deque()       # submitted, not admitted
        self.queue = collections.deque()         # bands of admitted jobs, not launched
        self.in_flight = []                      # launches on the device
        self.done = []                           # finished jobs
        self.cancelled = []                      # cancelled jobs, once nothing of theirs runs
        self.mem_in_use = 0
        self.lock = threading.Lock()
        self.next_ticket = 0
        self.launches = 0
        self.rejected = 0
        self.resident = {name: v.device_bytes() for name, v in volumes.items()}

    def resident_bytes(self) -> int:
        """Device bytes the resident cubes hold (all owners)."""
        return sum(a + b for a, b in self.resident.values())

    # -- client side ---------------------------------------------------------
    def submit(self, job: RenderJob) -> int:
        if job.cube not in self.volumes:
            raise KeyError("unknown cube %r" % job.cube)
        if job.out_bytes > self.mem_budget:
            self.rejected += 1
            raise ValueError("request needs %d bytes, more than the whole budget" % job.out_bytes)
        with self.lock:
            job.arrival = time.monotonic()
            job.ticket = self.next_ticket
            self.next_ticket += 1
            self.pending.append(job)
        return job.ticket

    def cancel(self, ticket: int) -> bool:
        """Cancel a submitted request; False if it is unknown or finished.
        Bands already launched run out; the request is then listed in
        ``cancelled`` instead of ``done``."""
        with self.lock:
            for job in self.pending:
                if job.ticket == ticket:
                    self.pending.remove(job)
                    job.cancelled = True
                    self.cancelled.append(job)
                    return True
            jobs = {u.job.ticket: u.job for u in self.queue}
            for ln in self.in_flight:
                for u in ln.units:
                    jobs.setdefault(u.job.ticket, u.job)
            job = jobs.get(ticket)
            if job is None or job.cancelled:
                return False
            job.cancelled = True
            dropped = [u for u in self.queue if u.job is job]
            for u in dropped:
                self.queue.remove(u)
            job.units -= len(dropped)
            self._retire_if_complete(job)
            return True

    # -- server side ---------------------------------------------------------
    def _admit(self):
        with self.lock:
            while self.pending and len(self.queue) < self.max_batch:
                job = self.pending[0]
                if self.mem_in_use + job.out_bytes > self.mem_budget:
                    break                          # first come, first served
                self.pending.popleft()
                self.mem_in_use += job.out_bytes
                job.admitted = time.monotonic()
                bands = plan_bands(job.h, job.w, self.band_rays)
                job.units = len(bands)
                for row0, rows in bands:
                    self.queue.append(_Unit(job, row0, rows))

    def _launch(self):
        if not self.queue or not self.free_streams:
            return False
        si = self.free_streams.popleft()
        stream = self.streams[si]
        with self.lock:
            units = take_units(self.queue, self.max_batch, self.launch_rays)
        if self.per_request:
            with torch.cuda.stream(stream):
                for u in units:
                    job = u.job
                    vol = self.volumes[job.cube]
                    if job.tf is not None:
                        vol.set_transfer(*job.tf)
                    job.out = vol.render(np.asarray([job.cam]), job.w, job.h, job.mode,
                                         job.step, stream=stream)
                    job.launched += 1
                ev = torch.cuda.Event()
                ev.record(stream)
            self.in_flight.append(_Launch(units, stream, ev, None, time.monotonic()))
            self.launches += 1
            return True
        flags = torch.zeros(len(units), dtype=torch.int32).pin_memory()
        reqs = []
        with torch.cuda.stream(stream):
            for i, u in enumerate(units):
                job = u.job
                if job.out is None:
                    shape = ((job.h, job.w, 4) if MODES[job.mode] == VR_COMPOSITE
                             else (job.h, job.w))
                    job.out = torch.empty(shape, dtype=torch.float32, device="cuda")
                band = None if u.rows == job.h else (u.row0, u.rows)
                reqs.append(Request(self.volumes[job.cube], job.cam, job.w, job.h, job.mode,
                                    job.step, out=job.out[u.row0:u.row0 + u.rows], tf=job.tf,
                                    done=(flags, i), done_value=1, band=band))
                job.launched += 1
            render_batch(reqs, self.workspaces[si], stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.in_flight.append(_Launch(units, stream, ev, flags, time.monotonic()))
        self.launches += 1
        return True

    def _retire_if_complete(self, job: RenderJob):
        """A job leaves the server once every band handed to a launch has
        retired and no band waits in the queue (units counts what remains)."""
        if job.retired < job.launched or job.units > job.launched:
            return
        if job.finished == 0.0:
            job.finished = time.monotonic()
        self.mem_in_use -= job.out_bytes
        if not self.keep_outputs:
            job.out = None
        (self.cancelled if job.cancelled else self.done).append(job)

    def _reap(self):
        """Record bands whose completion word is set (a job finishes with its
        last band); free finished launches."""
        now = time.monotonic()
        still = []
        for ln in self.in_flight:
            finished = ln.event.query()
            f = ln.flags.numpy() if ln.flags is not None else None
            for i, u in enumerate(ln.units):
                if not u.seen and (finished or (f is not None and f[i] != 0)):
                    u.seen = True
                    u.job.seen += 1
                    if u.job.seen == u.job.units and u.job.finished == 0.0:
                        u.job.finished = now
            if finished:
                for u in ln.units:
                    u.job.retired += 1
                    with self.lock:
                        self._retire_if_complete(u.job)
                self.free_streams.append(self.streams.index(ln.stream))
            else:
                still.append(ln)
        self.in_flight = still

    def step(self):
        """One turn of the serving loop: reap, admit, launch."""
        self._reap()
        self._admit()
        self._launch()

    def idle(self):
        with self.lock:
            return not self.pending and not self.queue and not self.in_flight

    def drain(self, timeout: float = 120.0):
        t0 = time.monotonic()
        while not self.idle():
            self.step()
            if time.monotonic() - t0 > timeout:
                raise TimeoutError("server did not drain")


def latency_stats(jobs):
    lat = np.array([j.latency for j in jobs]) * 1000.0
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max())}


def run_poisson(server: Server, make_job, rate: float, duration: float, seed: int = 0):
    """Submit jobs at Poisson arrival times (``rate`` per second) for
    ``duration`` seconds of wall clock while serving them; returns the
    finished jobs and the wall time until the last one finished."""
    rng = np.random.default_rng(seed)
    t0 = time.monotonic()
    next_t = t0 + rng.exponential(1.0 / rate)
    n = 0
    while True:
        now = time.monotonic()
        while next_t <= now and next_t < t0 + duration:
            server.submit(make_job(n))
            n += 1
            next_t += rng.exponential(1.0 / rate)
        server.step()
        if now >= t0 + duration and server.idle():
            break
        if now - t0 > duration + 120.0:
            raise TimeoutError("serving did not finish")
    return server.done, time.monotonic() - t0, n
