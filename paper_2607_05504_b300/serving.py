"""Continuous-batching service for SIDM halo-evolution requests.

A request is one isolated halo (particles, power-of-two bins, dt_max,
cross-section model, seed) to be advanced by n_steps scattering steps.
Requests that arrive while others are on the GPU are admitted as soon as a
free segment of the device-resident particle range can hold them; every tick
runs ONE multi-halo scattering step (sidm_step_haloes) over all resident
requests, each at its own step counter and active set, so their work
overlaps on the device; finished requests retire and free their segment.

Because every halo of a batch is stepped exactly as it would be alone (its
own tree, start radius, random key and step counter -- see sidm.h), a
request's result does not depend on what else is resident.

Layers:
  SegmentMap  host logic: the context's particle range [0, capacity) as
              segments, each a resident request or a hole; first-fit
              placement, holes merged, the unused tail trimmed, and the last
              resident moved into a hole that holds it (the build work of a
              tick covers the used range, holes included).
  Scheduler   host logic only (FIFO queue, admission into free segments,
              retirement); no device access.
  GpuEngine   device state: ONE library context sized once for the memory
              budget.  Admission writes only the new request's particles
              into its segment (sidm_write_particles); retirement reads only
              the finished request's velocities (sidm_read_particles); a
              resident moves only to close a hole, device to device
              (sidm_move_particles).  The active mask of a tick is
              formed on the device from per-particle admission ticks and bin
              periods; the tick's update count is known on the host from each
              request's bin histogram, so a tick needs no device round trip.
  Server      the loop: arrivals -> admission -> one step of all resident
              haloes -> retirement, with per-request latency.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I
from . import sidm


@dataclass
class Request:
    rid: int
    particles: I.Particles
    bins: np.ndarray
    dt_max: float
    n_steps: int
    seed: int
    sigma_kind: int = sidm.SIGMA_CONST
    sigma0: float = 1.0
    w: float = 1.0
    arrival: float = 0.0
    # filled in by the service
    steps_done: int = 0
    admitted: float | None = None
    finished: float | None = None
    result_vel: np.ndarray | None = None
    segment: int | None = None        # first particle of the request's segment

    @property
    def n(self) -> int:
        return self.particles.n

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival

    def active_count(self, s: int) -> int:
        """Active particles at the request's step s (host arithmetic on its
        bin histogram: bin b is active every 2^(bmax - b) steps)."""
        if self.n == 0:
            return 0
        hist = np.bincount(self.bins.astype(np.int64))
        bmax = hist.shape[0] - 1
        return int(sum(int(c) for b, c in enumerate(hist) if c and s % (1 << (bmax - b)) == 0))

    def active_counts(self) -> np.ndarray:
        """active_count(s) for every step s < n_steps, at once."""
        if self.n == 0:
            return np.zeros(self.n_steps, np.int64)
        hist = np.bincount(self.bins.astype(np.int64))
        bmax = hist.shape[0] - 1
        s = np.arange(self.n_steps, dtype=np.int64)[:, None]
        period = np.left_shift(np.int64(1), bmax - np.arange(hist.shape[0], dtype=np.int64))
        return ((s % period[None, :]) == 0).astype(np.int64) @ hist.astype(np.int64)


class SegmentMap:
    """The particle range [0, capacity) of one context as contiguous
    segments: resident requests (owner = request id) and holes (owner None).
    `end` is the used extent; segments cover [0, end) exactly."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.segs: list[list] = []        # [start, n, owner], sorted by start
        self.end = 0

    def place(self, n: int, owner) -> int | None:
        """First fit: the lowest hole that holds n particles, else the tail;
        None if neither can."""
        for k, (st, m, own) in enumerate(self.segs):
            if own is None and m >= n:
                if m > n:
                    self.segs.insert(k + 1, [st + n, m - n, None])
                self.segs[k] = [st, n, owner]
                return st
        if self.end + n <= self.capacity:
            st = self.end
            self.segs.append([st, n, owner])
            self.end += n
            return st
        return None

    def release(self, start: int) -> None:
        """Turns the segment at `start` into a hole, merges it with hole
        neighbours and trims a hole at the end of the used range."""
        k = next(i for i, s in enumerate(self.segs) if s[0] == start)
        self.segs[k][2] = None
        if k + 1 < len(self.segs) and self.segs[k + 1][2] is None:
            self.segs[k][1] += self.segs[k + 1][1]
            del self.segs[k + 1]
        if k > 0 and self.segs[k - 1][2] is None:
            self.segs[k - 1][1] += self.segs[k][1]
            del self.segs[k]
        while self.segs and self.segs[-1][2] is None:
            self.end -= self.segs[-1][1]
            self.segs.pop()

    def compact(self) -> list:
        """Closes holes: while the last segment (a resident, since a hole at
        the end is trimmed) fits into a hole before it, it moves into the
        lowest such hole.  Returns the moves as (owner, old start, new
        start, n), in order."""
        moves = []
        while len(self.segs) > 1:
            st, m, own = self.segs[-1]
            k = next((i for i, (hs, hm, ho) in enumerate(self.segs[:-1])
                      if ho is None and hm >= m), None)
            if k is None:
                break
            new = self.segs[k][0]
            hole_n = self.segs[k][1]
            self.segs[k] = [new, m, own]
            if hole_n > m:
                self.segs.insert(k + 1, [new + m, hole_n - m, None])
            self.release(st)
            moves.append((own, st, new, m))
        return moves

    def offsets(self) -> np.ndarray:
        off = np.zeros(len(self.segs) + 1, np.int64)
        off[1:] = np.cumsum([s[1] for s in self.segs]) if self.segs else []
        return off

    @property
    def free(self) -> int:
        return self.capacity - sum(s[1] for s in self.segs if s[2] is not None)


class Scheduler:
    """FIFO admission into free segments of a particle range sized by the
    device-memory budget (bytes) at `bytes_per_particle`."""

    def __init__(self, budget_bytes: float, bytes_per_particle: float):
        self.budget = float(budget_bytes)
        self.per_particle = float(bytes_per_particle)
        self.map = SegmentMap(int(self.budget // self.per_particle))
        self.queue: collections.deque[Request] = collections.deque()
        self.resident: list[Request] = []

    def cost(self, r: Request) -> float:
        return r.n * self.per_particle

    @property
    def used(self) -> float:
        return sum(self.cost(r) for r in self.resident)

    def submit(self, r: Request) -> None:
        if r.n > self.map.capacity:
            raise ValueError(f"request {r.rid} needs {self.cost(r):.3g} B > budget {self.budget:.3g} B")
        self.queue.append(r)

    def admit(self, now: float) -> list[Request]:
        """Admits queued requests in arrival order while each finds a segment."""
        new = []
        while self.queue:
            r = self.queue[0]
            st = self.map.place(r.n, r.rid)
            if st is None:
                break
            self.queue.popleft()
            r.segment = st
            r.admitted = now
            self.resident.append(r)
            new.append(r)
        return new

    def retire(self, now: float) -> list[Request]:
        done = [r for r in self.resident if r.steps_done >= r.n_steps]
        for r in done:
            r.finished = now
            self.map.release(r.segment)
        self.resident = [r for r in self.resident if r.steps_done < r.n_steps]
        return done

    def compact(self) -> list:
        """Moves resident requests from the end of the range into holes (see
        SegmentMap.compact); returns (request, old start, new start)."""
        by_id = {r.rid: r for r in self.resident}
        out = []
        for own, old, new, _ in self.map.compact():
            r = by_id[own]
            r.segment = new
            out.append((r, old, new))
        return out

    def layout(self) -> list:
        """Segments of the used range: (start, n, request or None)."""
        by_id = {r.rid: r for r in self.resident}
        return [(st, m, by_id.get(own) if own is not None else None)
                for st, m, own in self.map.segs]

    @property
    def idle(self) -> bool:
        return not self.queue and not self.resident


class GpuEngine:
    """Device side: one library context over the whole budget, resident
    requests in fixed segments."""

    HOLE_PERIOD = 1 << 62             # a hole particle is never active

    def __init__(self, budget_bytes: float, n_ngb: int = 64, device: int = 0, stream=None,
                 run_ahead: int = 2):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.dev)
        cfg = sidm.sidm_default_config()
        cfg.n_ngb = n_ngb
        self.bytes_per_particle = sidm.sidm_context_bytes(cfg, 1 << 20) / float(1 << 20)
        self.capacity = max(int(budget_bytes // self.bytes_per_particle), 64)
        self.ctx = sidm.Context(n_ngb=n_ngb, box=0.0, n_max=self.capacity, use_graph=True,
                                stream=self.stream.cuda_stream, device=device)
        z = np.zeros((0, 3))
        self.ctx.set_particles(z, z, np.zeros(0, np.uint32), mass_scalar=1.0)
        t = torch
        with t.cuda.stream(self.stream):
            self.bins = t.zeros(self.capacity, dtype=t.int8, device=self.dev)
            self.period = t.full((self.capacity,), self.HOLE_PERIOD, dtype=t.int64, device=self.dev)
            self.t0 = t.full((self.capacity,), -1, dtype=t.int64, device=self.dev)
        self.tick = 0
        self.layout: list = []
        self.params = None               # ctypes array of HaloParams, one per segment
        self.resident_k: list = []       # (segment index, request) of the resident requests
        self.counts: dict = {}           # request id -> active particles at each of its steps
        self.run_ahead = run_ahead
        self.events: collections.deque = collections.deque()

    def admit(self, reqs: list[Request], layout: list) -> None:
        """Writes each new request into its segment (nothing else moves)."""
        t = self.torch
        for r in reqs:
            p, st = r.particles, r.segment
            self.counts[r.rid] = r.active_counts()
            self.ctx.write_particles(st, p.pos, p.vel, p.ids, mass=p.mass)
            bmax = int(r.bins.max()) if r.n else 0
            with t.cuda.stream(self.stream):
                b = t.from_numpy(r.bins.astype(np.int8)).to(self.dev, non_blocking=False)
                self.bins[st:st + r.n].copy_(b)
                self.period[st:st + r.n] = t.bitwise_left_shift(
                    t.ones(r.n, dtype=t.int64, device=self.dev), bmax - b.to(t.int64))
                self.t0[st:st + r.n] = self.tick
        self.relayout(layout)

    def move(self, moves: list) -> None:
        """Moves resident requests to new segments, on the device (their
        particles, bins and step phases; their results do not change)."""
        t = self.torch
        for r, old, new in moves:
            self.ctx.move_particles(old, new, r.n)
            with t.cuda.stream(self.stream):
                for a in (self.bins, self.period, self.t0):
                    a[new:new + r.n].copy_(a[old:old + r.n].clone())

    def relayout(self, layout: list) -> None:
        """Haloes of the context = the segments (holes are haloes whose
        particles are never active)."""
        t = self.torch
        self.layout = layout
        end = layout[-1][0] + layout[-1][1] if layout else 0
        if end < self.ctx.n:
            self.ctx.set_count(end)
        for st, m, r in layout:
            if r is None:
                with t.cuda.stream(self.stream):
                    self.period[st:st + m] = self.HOLE_PERIOD
                    self.t0[st:st + m] = -1
        if end > 0:
            off = np.zeros(len(layout) + 1, np.int64)
            off[1:] = np.cumsum([m for _, m, _ in layout])
            self.ctx.set_haloes(off)
        hole = sidm.HaloParams(1.0, sidm.SigmaModel(sidm.SIGMA_CONST, 0.0, 1.0, 0.0), 0, 0)
        self.params = (sidm.HaloParams * max(len(layout), 1))(
            *[hole if r is None else
              sidm.HaloParams(r.dt_max, sidm.SigmaModel(r.sigma_kind, r.sigma0, r.w, 0.0),
                              r.seed, 0) for _, _, r in layout])
        self.resident_k = [(k, r) for k, (_, _, r) in enumerate(layout) if r is not None]
        live = {r.rid for _, r in self.resident_k}
        for rid in [rid for rid in self.counts if rid not in live]:
            del self.counts[rid]

    def step(self) -> int:
        """One scattering step of every resident request; returns the number
        of active particles (particle updates) of the tick, counted on the host."""
        t = self.torch
        if not self.layout:
            return 0
        end = self.ctx.n
        n_active = 0
        params = self.params
        for k, r in self.resident_k:
            params[k].step = r.steps_done
            n_active += int(self.counts[r.rid][r.steps_done])
        while len(self.events) >= self.run_ahead:     # bound the host's lead
            self.events.popleft().synchronize()
        with t.cuda.stream(self.stream):
            active = (t.remainder(self.tick - self.t0[:end], self.period[:end]) == 0).to(t.uint8)
        sidm._check(sidm.lib().sidm_step_haloes(self.ctx.handle, active.data_ptr(),
                                                self.bins[:end].data_ptr(), params, None),
                    "sidm_step_haloes")
        ev = t.cuda.Event()
        ev.record(self.stream)
        self.events.append(ev)
        self.tick += 1
        for _, r in self.resident_k:
            r.steps_done += 1
        return n_active

    def collect(self, done: list[Request]) -> None:
        """Copies the final velocities of finished requests to the host
        (their segments only)."""
        for r in done:
            r.result_vel = self.ctx.read_velocities(r.segment, r.n)

    def sync(self) -> int:
        return self.ctx.sync()

    def close(self) -> None:
        self.ctx.close()


@dataclass
class ServeReport:
    requests: int = 0
    ticks: int = 0
    updates: int = 0
    wall: float = 0.0
    latencies: list = field(default_factory=list)

    @property
    def throughput(self) -> float:
        return self.updates / self.wall if self.wall > 0 else 0.0

    def percentile(self, q: float) -> float:
        return float(np.percentile(self.latencies, q)) if self.latencies else math.nan


class Server:
    def __init__(self, engine, scheduler: Scheduler, clock=time.perf_counter, compact=True):
        """compact: after a retirement, move resident requests from the end of
        the range into the holes it left (the step's build work follows the
        used range, holes included)."""
        self.engine = engine
        self.sched = scheduler
        self.clock = clock
        self.compact = compact

    def run(self, requests: list[Request], max_ticks: int = 10 ** 9) -> ServeReport:
        """Serves requests whose .arrival are offsets (s) from the start."""
        pending = sorted(requests, key=lambda r: r.arrival)
        rep = ServeReport(requests=len(requests))
        t0 = self.clock()
        i = 0
        while (i < len(pending) or not self.sched.idle) and rep.ticks < max_ticks:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                self.sched.submit(pending[i])
                i += 1
            if self.sched.idle:
                # nothing to do before the next arrival
                time.sleep(max(0.0, min(pending[i].arrival - now, 0.01)))
                continue
            new = self.sched.admit(now)
            if new:
                self.engine.admit(new, self.sched.layout())
            rep.updates += self.engine.step()
            rep.ticks += 1
            done = [r for r in self.sched.resident if r.steps_done >= r.n_steps]
            if done:
                self.engine.collect(done)
                self.sched.retire(self.clock() - t0)
                if self.compact:
                    moves = self.sched.compact()
                    if moves:
                        self.engine.move(moves)
                self.engine.relayout(self.sched.layout())
        self.engine.sync()
        rep.wall = self.clock() - t0
        rep.latencies = [r.latency for r in requests if r.latency is not None]
        return rep


def request_stream(n_req: int, rate: float, seed: int = 3, log2_n=(12.0, 21.0),
                   steps=(10, 1000), pool: int = 0, n_ngb: int = 64) -> list[Request]:
    """Poisson arrivals (rate per second) of halo requests: N log-uniform in
    2^[log2_n], Hernquist or NFW with p = 1/2, constant or Yukawa-like sigma
    with p = 1/2, sigma0/m log-uniform in [0.1, 10], steps log-uniform in
    [steps].  pool = 0: every request is its own halo (its own size and
    seed); pool > 0: sizes are quantised to `pool` log-spaced values and the
    particle sets of equal size and profile are shared (faster to generate;
    each request still has its own seed, cross-section and step count)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    sizes = np.round(2.0 ** rng.uniform(log2_n[0], log2_n[1], n_req)).astype(np.int64)
    grid = (np.unique(np.round(np.geomspace(2 ** log2_n[0], 2 ** log2_n[1], pool)).astype(np.int64))
            if pool > 0 else None)
    cache: dict = {}
    out = []
    for k in range(n_req):
        if grid is not None:
            nq = int(grid[np.argmin(np.abs(np.log(grid) - math.log(sizes[k])))])
        else:
            nq = int(sizes[k])
        prof = "hernquist" if rng.random() < 0.5 else "nfw"
        key = (prof, nq) if grid is not None else (prof, nq, k)
        if key not in cache:
            hs = 11 + nq if grid is not None else 100003 * (k + 1) + seed
            p = I.hernquist_halo(nq, hs) if prof == "hernquist" else I.nfw_halo(nq, hs + 2)
            dens = I.hernquist_density if prof == "hernquist" else I.nfw_density
            cache[key] = (p, dens)
        p, dens = cache[key]
        yuk = rng.random() < 0.5
        s0 = float(10 ** rng.uniform(-1, 1))
        w = float(p.meta.get("v_c_rs", 0.7)) if yuk else 1.0
        bins, dt = I.timestep_bins(p, dens, s0, n_ngb)
        out.append(Request(rid=k, particles=p, bins=bins, dt_max=dt,
                           n_steps=int(round(10 ** rng.uniform(math.log10(steps[0]), math.log10(steps[1])))),
                           seed=int(rng.integers(0, 2 ** 63)), sigma_kind=int(yuk), sigma0=s0, w=w,
                           arrival=float(arrivals[k])))
    return out
