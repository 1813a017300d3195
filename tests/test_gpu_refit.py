"""Tree reuse between full rebuilds (rebuild_every > 1): the steps in between
keep the last key order and refit the boxes to the current positions.  The
results must not change while particles drift between steps: every step
equals the oracle's, with and without graph replay."""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _drift_run(ctx, p, bins, dt_max, steps, drift):
    pos, vel = p.pos.copy(), p.vel.copy()
    out = []
    for k in range(steps):
        act = I.active_at_step(bins, k)
        ctx.set_particles(pos, vel, p.ids, mass=p.mass)
        ctx.step_counter = k
        ctx.step(dt_max, act, bins, seed=21, stats=False)
        vel, h = ctx.velocities()
        out.append((pos.copy(), vel.copy(), h, ctx.timestep_limits(), ctx.pairs()))
        pos = pos + drift * vel          # positions move between steps
    return out


@pytest.mark.parametrize("use_graph", [False, True])
def test_refit_steps_equal_the_oracle_while_particles_drift(use_graph):
    p = I.hernquist_halo(12000, 14, ids="random")
    bins = np.random.default_rng(3).integers(0, 3, p.n).astype(np.int8)
    ctx = sidm.Context(n_ngb=32, rebuild_every=4, use_graph=use_graph)
    res = _drift_run(ctx, p, bins, 1.0, 9, drift=0.05)
    ctx.close()
    for k, (pos, vel_after, gh, gl, (ab, ords)) in enumerate(res):
        vel_before = p.vel if k == 0 else res[k - 1][1]
        # set_particles starts every step with h = 0 and dt_lim = inf
        o = oracle.step(pos, vel_before, p.mass, p.ids, I.active_at_step(bins, k), bins, 1.0,
                        n_ngb=32, seed=21, step=k)
        assert np.array_equal(gh, o["h"]), k
        assert np.array_equal(ab, o["pairs_ab"][: o["n_pairs"]]), k
        assert np.array_equal(ords, o["pairs_ord"][: o["n_pairs"]]), k
        assert np.array_equal(vel_after, o["vel"]), k
        assert np.array_equal(gl, o["dtlim"]), k


def test_refit_equals_rebuild_every_step():
    p = I.hernquist_halo(30000, 15)
    bins = np.random.default_rng(4).integers(0, 4, p.n).astype(np.int8)
    a = sidm.Context(n_ngb=64)
    b = sidm.Context(n_ngb=64, rebuild_every=6, use_graph=True)
    ra = _drift_run(a, p, bins, 1.0, 12, drift=0.02)
    rb = _drift_run(b, p, bins, 1.0, 12, drift=0.02)
    a.close()
    b.close()
    for x, y in zip(ra, rb):
        for u, v in zip(x[1:4], y[1:4]):
            assert np.array_equal(u, v)
        assert np.array_equal(x[4][0], y[4][0]) and np.array_equal(x[4][1], y[4][1])
