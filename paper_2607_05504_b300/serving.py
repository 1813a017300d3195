"""Continuous-batching service for SIDM halo-evolution requests.

A request is one isolated halo (particles, power-of-two bins, dt_max,
cross-section model, seed) to be advanced by n_steps scattering steps.
Requests that arrive while others are on the GPU are admitted as soon as the
device-memory budget allows; every tick runs ONE multi-halo scattering step
(sidm_step_haloes) over all resident requests, each at its own step counter
and active set, so their work overlaps on the device; finished requests
retire and free their share of the budget.

Because every halo of a batch is stepped exactly as it would be alone (its
own tree, start radius, random key and step counter -- see sidm.h), a
request's result does not depend on what else is resident.

Layers:
  Scheduler  host logic only (queue, FIFO admission under the budget,
             retirement); no device access.
  GpuEngine  device state: each resident request's arrays as device tensors,
             packed into one library context whenever the resident set
             changes; the active mask of a tick is formed on the device.
  Server     the loop: arrivals -> admission -> one step of all resident
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

    @property
    def n(self) -> int:
        return self.particles.n

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


class Scheduler:
    """FIFO admission under a device-memory budget (bytes)."""

    def __init__(self, budget_bytes: float, bytes_per_particle: float):
        self.budget = float(budget_bytes)
        self.per_particle = float(bytes_per_particle)
        self.queue: collections.deque[Request] = collections.deque()
        self.resident: list[Request] = []
        self.used = 0.0

    def cost(self, r: Request) -> float:
        return r.n * self.per_particle

    def submit(self, r: Request) -> None:
        if self.cost(r) > self.budget:
            raise ValueError(f"request {r.rid} needs {self.cost(r):.3g} B > budget {self.budget:.3g} B")
        self.queue.append(r)

    def admit(self, now: float) -> list[Request]:
        """Admits queued requests in arrival order while they fit."""
        new = []
        while self.queue and self.used + self.cost(self.queue[0]) <= self.budget:
            r = self.queue.popleft()
            r.admitted = now
            self.used += self.cost(r)
            self.resident.append(r)
            new.append(r)
        return new

    def retire(self, now: float) -> list[Request]:
        done = [r for r in self.resident if r.steps_done >= r.n_steps]
        for r in done:
            r.finished = now
            self.used -= self.cost(r)
        self.resident = [r for r in self.resident if r.steps_done < r.n_steps]
        return done

    @property
    def idle(self) -> bool:
        return not self.queue and not self.resident


class GpuEngine:
    """Device side: one library context over the resident requests."""

    def __init__(self, capacity: int, n_ngb: int = 64, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.dev)
        self.ctx = sidm.Context(n_ngb=n_ngb, box=0.0, n_max=max(int(capacity), 64),
                                stream=self.stream.cuda_stream, device=device)
        self.resident: list[Request] = []
        self.dev_state: dict[int, dict] = {}
        self.off = np.zeros(1, np.int64)

    def _upload(self, r: Request) -> dict:
        t = self.torch
        p = r.particles
        with t.cuda.stream(self.stream):
            return {"pos": t.from_numpy(p.pos).to(self.dev), "vel": t.from_numpy(p.vel).to(self.dev),
                    "mass": t.from_numpy(p.mass).to(self.dev),
                    "ids": t.from_numpy(p.ids.view(np.int32)).to(self.dev),
                    "bins": t.from_numpy(r.bins.astype(np.int8)).to(self.dev),
                    "bmax": int(r.bins.max()) if r.n else 0}

    def _save_velocities(self) -> None:
        """Current velocities of the resident requests back into their tensors."""
        if not self.resident or self.off[-1] == 0:
            return
        t = self.torch
        v = t.empty((int(self.off[-1]), 3), dtype=t.float64, device=self.dev)
        sidm.sidm_get_particles(self.ctx.handle, v)
        with t.cuda.stream(self.stream):
            for k, r in enumerate(self.resident):
                self.dev_state[r.rid]["vel"].copy_(v[self.off[k]:self.off[k + 1]])

    def set_resident(self, reqs: list[Request]) -> None:
        t = self.torch
        self._save_velocities()
        for r in reqs:
            if r.rid not in self.dev_state:
                self.dev_state[r.rid] = self._upload(r)
        for rid in [rid for rid in self.dev_state if rid not in {r.rid for r in reqs}]:
            del self.dev_state[rid]
        self.resident = list(reqs)
        sizes = [r.n for r in reqs]
        self.off = np.zeros(len(reqs) + 1, np.int64)
        self.off[1:] = np.cumsum(sizes)
        if not reqs:
            return
        S = [self.dev_state[r.rid] for r in reqs]
        with t.cuda.stream(self.stream):
            self.pos = t.cat([s["pos"] for s in S])
            self.vel = t.cat([s["vel"] for s in S])
            self.mass = t.cat([s["mass"] for s in S])
            self.ids = t.cat([s["ids"] for s in S])
            self.bins = t.cat([s["bins"] for s in S])
            sz = t.tensor(sizes, device=self.dev)
            self.bmax_p = t.repeat_interleave(t.tensor([s["bmax"] for s in S], device=self.dev), sz)
            self.steps_p = t.repeat_interleave(
                t.tensor([r.steps_done for r in reqs], dtype=t.int64, device=self.dev), sz)
            self.period_p = t.bitwise_left_shift(t.ones_like(self.bmax_p),
                                                 self.bmax_p - self.bins.to(t.int64))
        self.ctx.set_particles(self.pos, self.vel, self.ids, mass=self.mass)
        self.ctx.set_haloes(self.off)

    def step(self) -> int:
        """One scattering step of every resident request; returns the number
        of active particles (particle updates) of the tick."""
        t = self.torch
        if not self.resident:
            return 0
        with t.cuda.stream(self.stream):
            active = (t.remainder(self.steps_p, self.period_p) == 0).to(t.uint8)
            n_active = int(active.sum().item())
        params = [sidm.HaloParams(r.dt_max, sidm.SigmaModel(r.sigma_kind, r.sigma0, r.w),
                                  r.seed, r.steps_done) for r in self.resident]
        sidm.sidm_step_haloes(self.ctx.handle, active, self.bins, params, None)
        with t.cuda.stream(self.stream):
            self.steps_p += 1
        for r in self.resident:
            r.steps_done += 1
        return n_active

    def collect(self, done: list[Request]) -> None:
        """Copies the final velocities of finished requests to the host."""
        if not done:
            return
        self._save_velocities()
        for r in done:
            r.result_vel = self.dev_state[r.rid]["vel"].cpu().numpy()

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
    def __init__(self, engine, scheduler: Scheduler, clock=time.perf_counter):
        self.engine = engine
        self.sched = scheduler
        self.clock = clock

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
                self.engine.set_resident(self.sched.resident)
            rep.updates += self.engine.step()
            rep.ticks += 1
            done = [r for r in self.sched.resident if r.steps_done >= r.n_steps]
            if done:
                self.engine.collect(done)
                self.sched.retire(self.clock() - t0)
                self.engine.set_resident(self.sched.resident)
        self.engine.sync()
        rep.wall = self.clock() - t0
        rep.latencies = [r.latency for r in requests if r.latency is not None]
        return rep


def request_stream(n_req: int, rate: float, seed: int = 3, log2_n=(12.0, 21.0),
                   steps=(10, 1000), pool: int = 16, n_ngb: int = 64) -> list[Request]:
    """Poisson arrivals (rate per second) of halo requests: N log-uniform in
    2^[log2_n], Hernquist or NFW with p = 1/2, constant or Yukawa-like sigma
    with p = 1/2, sigma0/m log-uniform in [0.1, 10], steps log-uniform in
    [steps].  Particle sets come from a pool of `pool` generated haloes per
    profile (each request has its own seed, cross-section and step count)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    sizes = np.round(2.0 ** rng.uniform(log2_n[0], log2_n[1], n_req)).astype(np.int64)
    # quantise sizes to the pool (log-spaced) so that haloes can be reused
    grid = np.unique(np.round(np.geomspace(2 ** log2_n[0], 2 ** log2_n[1], pool)).astype(np.int64))
    cache: dict = {}
    out = []
    for k in range(n_req):
        nq = int(grid[np.argmin(np.abs(np.log(grid) - math.log(sizes[k])))])
        prof = "hernquist" if rng.random() < 0.5 else "nfw"
        key = (prof, nq)
        if key not in cache:
            p = I.hernquist_halo(nq, 11 + nq) if prof == "hernquist" else I.nfw_halo(nq, 13 + nq)
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
