"""sidm_set_positions: new positions between steps with everything else
kept (masses, ids, h and the Eq. 18 limits of inactive particles, the halo
layout, the kept key order).  Every step must equal the oracle's step on the
same state, with tree reuse and graph replay."""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("use_graph,rebuild_every", [(False, 1), (True, 4)])
def test_drifting_positions_match_the_oracle(use_graph, rebuild_every):
    p = I.hernquist_halo(12000, 31, ids="random")
    bins = np.random.default_rng(32).integers(0, 3, p.n).astype(np.int8)
    ctx = sidm.Context(n_ngb=32, use_graph=use_graph, rebuild_every=rebuild_every)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    pos, vel = p.pos.copy(), p.vel.copy()
    h = np.zeros(p.n)
    dl = np.full(p.n, np.inf)
    for k in range(7):
        act = I.active_at_step(bins, k)
        ctx.step(1.0, act, bins, seed=33, stats=False)
        gv, gh = ctx.velocities()
        gl = ctx.timestep_limits()
        o = oracle.step(pos, vel, p.mass, p.ids, act, bins, 1.0, n_ngb=32, seed=33, step=k,
                        h_init=h, dtlim_init=dl)
        assert np.array_equal(gh, o["h"]), k
        assert np.array_equal(gl, o["dtlim"]), k
        assert np.array_equal(gv, o["vel"]), k
        ab, ords = ctx.pairs()
        assert np.array_equal(ab, o["pairs_ab"][: o["n_pairs"]]), k
        assert np.array_equal(ords, o["pairs_ord"][: o["n_pairs"]]), k
        vel, h, dl = o["vel"], o["h"], o["dtlim"]
        # the particles drift; a gravity solver would also change the velocities
        pos = pos + 0.03 * vel
        vel = vel * 0.999
        ctx.set_positions(pos)
        ctx.set_velocities(vel)
    ctx.close()


def test_positions_outside_the_periodic_box_are_rejected():
    p = I.uniform_box(2000, 1.0, 1.0, 34)
    ctx = sidm.Context(box=1.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    good = p.pos.copy()
    good[:, 0] = (good[:, 0] + 0.25) % 1.0
    good[good >= 1.0] = 0.0
    ctx.set_positions(good)
    bad = good.copy()
    bad[7, 2] = 1.0
    with pytest.raises(sidm.SidmError) as e:
        ctx.set_positions(bad)
    assert e.value.status == sidm.ERR_INVALID_ARG
    ctx.close()


def test_velocity_uploads_are_ordered_with_every_use():
    """sidm_set_velocities copies beside the context's stream; every later
    use (a read-back, a step, another upload) sees the newest values."""
    p = I.uniform_box(5000, 1.0, 1.0, 35, ids="random")
    bins = np.zeros(p.n, np.int8)
    rng = np.random.default_rng(36)
    v1, v2 = rng.normal(size=p.vel.shape), rng.normal(size=p.vel.shape)
    for use_graph in (False, True):
        ctx = sidm.Context(box=1.0, use_graph=use_graph)
        ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
        ctx.step(0.1, None, bins, seed=37, stats=False)
        ctx.set_velocities(v1)
        assert np.array_equal(ctx.velocities()[0], v1)
        ctx.set_velocities(v2)
        ctx.set_velocities(v1)
        ctx.step(0.1, None, bins, seed=37, stats=False)
        o = oracle.step(p.pos, v1, p.mass, p.ids, None, bins, 0.1, box=1.0, seed=37, step=1)
        assert np.array_equal(ctx.velocities()[0], o["vel"]), use_graph
        ctx.close()
