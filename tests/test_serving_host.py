"""Host logic of the continuous-batching service (no GPU): admission in
arrival order into free segments of the budget's particle range, admission
of waiting requests as segments free up, retirement after n_steps, hole
merging, latency bookkeeping."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import serving as S


class FakeEngine:
    def __init__(self):
        self.resident_history = []
        self.steps = 0
        self.layout = []
        self.writes = []
        self.moves = []

    def admit(self, reqs, layout):
        self.writes += [(r.rid, r.segment, r.n) for r in reqs]
        self.relayout(layout)

    def relayout(self, layout):
        self.layout = list(layout)
        self.resident_history.append([r.rid for _, _, r in layout if r is not None])
        # segments tile [0, end) in order
        pos = 0
        for st, m, _ in layout:
            assert st == pos
            pos += m

    def move(self, moves):
        self.moves += [(r.rid, old, new) for r, old, new in moves]

    def step(self):
        self.steps += 1
        res = [r for _, _, r in self.layout if r is not None]
        for r in res:
            r.steps_done += 1
        return sum(r.n for r in res)

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


def test_segment_map_first_fit_merge_and_trim():
    m = S.SegmentMap(1000)
    assert m.place(300, "a") == 0 and m.place(300, "b") == 300 and m.place(300, "c") == 600
    assert m.place(200, "x") is None                     # 100 left at the tail
    m.release(300)                                       # hole [300, 600) in the middle
    assert m.end == 900 and m.free == 400
    assert m.place(200, "d") == 300                      # first fit: into the hole
    assert [s[2] for s in m.segs] == ["a", "d", None, "c"]
    assert m.place(250, "e") is None                     # 100 + 100 apart: no fit
    m.release(600)                                       # c: merges with the hole, then trimmed
    assert m.end == 500 and [s[2] for s in m.segs] == ["a", "d"]
    assert m.place(250, "e") == 500
    m.release(0)
    m.release(300)                                       # d: merges with a's hole on the left
    assert [(s[0], s[1], s[2]) for s in m.segs] == [(0, 500, None), (500, 250, "e")]
    assert list(m.offsets()) == [0, 500, 750]
    m.release(500)
    assert m.end == 0 and m.segs == [] and m.free == 1000


def test_compaction_moves_the_last_resident_into_the_lowest_hole():
    m = S.SegmentMap(1000)
    for o, n in (("a", 300), ("b", 200), ("c", 100), ("d", 150)):
        m.place(n, o)
    m.release(0)                                         # a: hole [0, 300)
    # d into the hole (the tail trims), then c into what is left of it
    assert m.compact() == [("d", 600, 0, 150), ("c", 500, 150, 100)]
    assert [(s[0], s[1], s[2]) for s in m.segs] == [(0, 150, "d"), (150, 100, "c"),
                                                    (250, 50, None), (300, 200, "b")]
    assert m.end == 500 and m.compact() == []            # b does not fit into 50


def test_resident_requests_move_only_to_close_holes():
    reqs = [_req(0, 400, 2, 0.0), _req(1, 300, 6, 0.0), _req(2, 200, 3, 0.0),
            _req(3, 350, 2, 0.05)]
    eng = FakeEngine()
    S.Server(eng, S.Scheduler(1000.0, 1.0), clock=FakeClock()).run(reqs)
    # the only moves are into holes below the mover's old segment
    assert all(new < old for _, old, new in eng.moves)
    assert all(r.result_vel is not None for r in reqs)


def test_resident_requests_never_move_without_compaction():
    reqs = [_req(0, 400, 2, 0.0), _req(1, 300, 6, 0.0), _req(2, 200, 3, 0.0),
            _req(3, 350, 2, 0.05)]
    eng = FakeEngine()
    S.Server(eng, S.Scheduler(1000.0, 1.0), clock=FakeClock(), compact=False).run(reqs)
    assert eng.moves == []
    # each request was written once, at its segment, and kept it while resident
    assert sorted(w[0] for w in eng.writes) == [0, 1, 2, 3]
    seg = {w[0]: w[1] for w in eng.writes}
    assert seg[1] == 400                                 # behind request 0
    assert seg[3] == 0                                   # into the hole request 0 left
    assert all(r.result_vel is not None for r in reqs)


def test_active_count_from_bins():
    r = _req(0, 64, 5, 0.0)
    r.bins = np.array([0] * 10 + [1] * 20 + [3] * 34, np.int8)
    for s in range(9):
        assert r.active_count(s) == int(I.active_at_step(r.bins, s).sum())


def test_request_stream_recipe():
    rs = S.request_stream(40, rate=200.0, seed=3, log2_n=(10.0, 12.0), steps=(10, 1000), pool=4)
    arr = np.array([r.arrival for r in rs])
    assert np.all(np.diff(arr) >= 0) and 0.05 < arr[-1] < 1.0
    assert all(10 <= r.n_steps <= 1000 for r in rs)
    assert {r.sigma_kind for r in rs} == {0, 1}
    assert len({r.seed for r in rs}) == len(rs)
    assert all(2 ** 10 * 0.9 <= r.n <= 2 ** 12 * 1.1 for r in rs)
    own = S.request_stream(6, rate=200.0, seed=4, log2_n=(10.0, 12.0), steps=(10, 20))
    assert len({r.particles.pos[0, 0] for r in own}) == 6      # every request its own halo
