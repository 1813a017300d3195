"""Launch shapes and the captured step graph change only the time of a step:
results must be bit-identical to direct launches with the default shapes,
and the autotuner must leave the simulation state where it was."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _halo(n=1 << 14, seed=21):
    p = I.hernquist_halo(n, seed)
    bins, dt = I.timestep_bins(p, I.hernquist_density, 1.0, 64)
    return p, bins, dt


def _run(p, bins, dt, steps, **ctx_kw):
    tune = ctx_kw.pop("tune", None)
    ctx = sidm.Context(n_ngb=64, **ctx_kw)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    if tune:
        ctx.set_tuning(**tune)
    out = []
    for s in range(steps):
        act = I.active_at_step(bins, s)
        ctx.step(dt, act, bins, seed=5, stats=False)
        v, h = ctx.velocities()
        out.append((v, h, ctx.timestep_limits(), ctx.pairs()[1]))
    state = ctx.graph_state
    ctx.close()
    return out, state


def _same(a, b):
    for (v1, h1, d1, o1), (v2, h2, d2, o2) in zip(a, b):
        assert np.array_equal(v1, v2)
        assert np.array_equal(h1, h2)
        assert np.array_equal(d1, d2)
        assert np.array_equal(o1, o2)


def test_graph_replay_is_bit_identical():
    p, bins, dt = _halo()
    ref, st0 = _run(p, bins, dt, 5)
    got, st1 = _run(p, bins, dt, 5, use_graph=True)
    assert st0 == 0
    assert st1 == 1          # the step ran as a captured graph
    _same(ref, got)


@pytest.mark.parametrize("tune", [
    dict(search_window=128, search_chunk=1, search_blocks_per_sm=4, pairs_chunk=16,
         pairs_blocks_per_sm=3),
    dict(search_window=512, search_chunk=16, search_blocks_per_sm=6, pairs_chunk=1,
         pairs_blocks_per_sm=4),
    dict(search_window=768, search_chunk=2),
    dict(search_window=1024, search_chunk=4, search_blocks_per_sm=8),
    # runs of consecutive queries per warp: each query after a run's first
    # sizes its gather from its predecessor's h (1: every query on its own)
    dict(search_run=1),
    dict(search_run=3, search_blocks_per_sm=2),
    dict(search_run=16, search_chunk=2, search_window=256),
])
def test_launch_shapes_do_not_change_results(tune):
    p, bins, dt = _halo(seed=22)
    ref, _ = _run(p, bins, dt, 3)
    got, _ = _run(p, bins, dt, 3, tune=tune)
    _same(ref, got)


def test_invalid_shapes_are_rejected():
    ctx = sidm.Context()
    before = ctx.tuning
    for bad in (dict(search_window=300), dict(search_chunk=65), dict(search_blocks_per_sm=9),
                dict(pairs_blocks_per_sm=8), dict(search_run=17)):
        with pytest.raises(sidm.SidmError) as e:
            ctx.set_tuning(**bad)
        assert e.value.status == sidm.ERR_INVALID_ARG
        assert ctx.tuning == before
    ctx.close()


def test_autotune_leaves_the_state_and_results_unchanged():
    p, bins, dt = _halo(seed=23)
    ref, _ = _run(p, bins, dt, 3)
    ctx = sidm.Context(n_ngb=64, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    prm = [sidm.HaloParams(dt, sidm.SigmaModel(0, 1.0, 1.0), 5, 0)]
    best = ctx.autotune(prm, I.active_at_step(bins, 0), bins, reps=2)
    assert best["search_window"] in (128, 256, 384, 512, 768, 1024)
    assert ctx.tuning == best
    assert ctx.step_counter == 0
    v, _ = ctx.velocities()
    assert np.array_equal(v, p.vel)
    got = []
    for s in range(3):
        ctx.step(dt, I.active_at_step(bins, s), bins, seed=5, stats=False)
        v, h = ctx.velocities()
        got.append((v, h, ctx.timestep_limits(), ctx.pairs()[1]))
    assert ctx.graph_state == 1
    ctx.close()
    _same(ref, got)


def test_graph_with_many_haloes_follows_their_step_counters():
    """Per-halo parameters change every tick (step counters, seeds); they are
    uploaded before each graph replay."""
    hs = I.hernquist_batch(6, seed=300, log2_n=(10, 13))
    p, off, bins = I.pack(hs)

    def run(use_graph):
        ctx = sidm.Context(n_ngb=64, use_graph=use_graph)
        ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
        ctx.set_haloes(off)
        res = []
        for s in range(4):
            act = np.concatenate([I.active_at_step(h["bins"], s) for h in hs])
            prm = [sidm.HaloParams(h["dt_max"], sidm.SigmaModel(0, h["sigma0"], 1.0), h["seed"],
                                   s + 3 * k) for k, h in enumerate(hs)]
            ctx.step_haloes(prm, act, bins, stats=False)
            res.append(ctx.velocities()[0])
        st = ctx.graph_state
        ctx.close()
        return res, st

    a, _ = run(False)
    b, st = run(True)
    assert st == 1
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
