"""Host logic of the continuous-batching service (no GPU): admission in
arrival order under the memory budget, admission of waiting requests as
memory frees up, retirement after n_steps, latency bookkeeping."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import serving as S


class FakeEngine:
    def __init__(self):
        self.resident_history = []
        self.steps = 0

    def set_resident(self, reqs):
        self.resident = list(reqs)
        self.resident_history.append([r.rid for r in reqs])

    def step(self):
        self.steps += 1
        for r in self.resident:
            r.steps_done += 1
        return sum(r.n for r in self.resident)

    def collect(self, done):
        for r in done:
            r.result_vel = np.zeros((r.n, 3))

    def sync(self):
        return 0


class FakeClock:
    def __init__(self, dt=0.01):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def _req(rid, n, steps, arrival):
    p = I.uniform_box(n, 1.0, 1.0, rid)
    return S.Request(rid=rid, particles=p, bins=np.zeros(n, np.int8), dt_max=0.1, n_steps=steps,
                     seed=rid, arrival=arrival)


def test_admission_budget_and_order():
    sch = S.Scheduler(budget_bytes=1000.0, bytes_per_particle=1.0)
    a, b, c = _req(0, 600, 3, 0.0), _req(1, 300, 2, 0.0), _req(2, 500, 1, 0.0)
    for r in (a, b, c):
        sch.submit(r)
    assert [r.rid for r in sch.admit(0.0)] == [0, 1]     # c does not fit yet
    assert sch.used == 900.0
    b.steps_done = 2
    assert [r.rid for r in sch.retire(1.0)] == [1]
    assert sch.admit(1.0) == []                          # 600 + 500 > 1000: still waits
    a.steps_done = 3
    sch.retire(2.0)
    assert [r.rid for r in sch.admit(2.0)] == [2]
    with pytest.raises(ValueError):
        sch.submit(_req(9, 2000, 1, 0.0))


def test_server_serves_every_request_and_overlaps_them():
    reqs = [_req(0, 400, 5, 0.0), _req(1, 300, 3, 0.015), _req(2, 500, 4, 0.02),
            _req(3, 200, 2, 0.03), _req(4, 100, 6, 0.5)]
    eng = FakeEngine()
    srv = S.Server(eng, S.Scheduler(900.0, 1.0), clock=FakeClock())
    rep = srv.run(reqs)
    assert all(r.steps_done == r.n_steps and r.result_vel is not None for r in reqs)
    assert rep.requests == 5 and len(rep.latencies) == 5
    # requests overlapped on the device (more than one resident at once)
    assert max(len(h) for h in eng.resident_history) >= 2
    # request 2 had to wait for memory (400 + 300 + 500 > 900)
    assert reqs[2].admitted > reqs[2].arrival
    assert all(r.finished >= r.admitted >= r.arrival for r in reqs)
    assert rep.percentile(50) <= rep.percentile(99)


def test_request_stream_recipe():
    rs = S.request_stream(40, rate=200.0, seed=3, log2_n=(10.0, 12.0), steps=(10, 1000), pool=4)
    arr = np.array([r.arrival for r in rs])
    assert np.all(np.diff(arr) >= 0) and 0.05 < arr[-1] < 1.0
    assert all(10 <= r.n_steps <= 1000 for r in rs)
    assert {r.sigma_kind for r in rs} == {0, 1}
    assert len({r.seed for r in rs}) == len(rs)
    assert all(2 ** 10 * 0.9 <= r.n <= 2 ** 12 * 1.1 for r in rs)
