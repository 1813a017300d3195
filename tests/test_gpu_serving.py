"""Continuous batching on the GPU: requests that arrive while others run are
admitted as memory frees up, their steps overlap in one multi-halo step per
tick, and each request's result is bit-identical to the request run alone."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import serving as S
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


class FakeClock:
    def __init__(self, dt=0.01):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def _alone(r: S.Request) -> np.ndarray:
    p = r.particles
    ctx = sidm.Context(n_ngb=64, box=0.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    for s in range(r.n_steps):
        ctx.step_counter = s
        ctx.step(r.dt_max, I.active_at_step(r.bins, s), r.bins, sigma0=r.sigma0,
                 sigma_kind=r.sigma_kind, w=r.w, seed=r.seed, stats=False)
    v, _ = ctx.velocities()
    ctx.close()
    return v


def test_each_request_is_the_same_alone_and_in_the_mix():
    reqs = S.request_stream(7, rate=60.0, seed=5, log2_n=(10.0, 13.5), steps=(3, 9), pool=4)
    biggest = max(r.n for r in reqs)
    probe = S.GpuEngine(budget_bytes=1e6)
    bpp = probe.bytes_per_particle
    probe.close()
    eng = S.GpuEngine(budget_bytes=2.2 * biggest * bpp)
    sched = S.Scheduler(budget_bytes=2.2 * biggest * bpp, bytes_per_particle=bpp)
    rep = S.Server(eng, sched, clock=FakeClock()).run(reqs)
    eng.close()
    assert rep.requests == 7 and len(rep.latencies) == 7
    assert any(r.admitted > r.arrival + 1e-9 for r in reqs)       # some waited for memory
    assert rep.updates == sum(sum(r.active_count(s) for s in range(r.n_steps)) for r in reqs)
    for r in reqs:
        assert r.result_vel is not None and r.steps_done == r.n_steps
        v = _alone(r)
        assert np.array_equal(r.result_vel, v), f"request {r.rid}"
        assert not np.array_equal(v, r.particles.vel)
