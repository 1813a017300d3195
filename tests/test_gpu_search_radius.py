"""The search's first gather radius from the h of a particle's last search
(the context's opt-in search hint; the plain form carries no h between
steps).

With the hint, a query whose particle has an h from an earlier step first
gathers within 9/8 of it, and keeps that radius only when K = N_ngb + tol +
1 gathered entries are surely inside; otherwise it takes the key-order
window's radius.
Either radius bounds the K-th neighbour, and the h bisection counts exactly
below it, so the result must be the oracle's whichever radius was used
(Sec. 4.2 and 4.5: the iterative h search).  These steps follow a first
step, so that the earlier h exists, with the positions kept, contracted
(the first radius holds many more particles than needed, or more than the
gather list holds, so the window takes over) or expanded (too few
particles inside: the window takes over)."""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

from test_gpu_parity import _compare, _gpu_step

pytestmark = pytest.mark.gpu


def _steps(p, positions, masks, bins, dt_max, *, n_ngb=32, seed=5, overlap_table=None):
    """Steps the context (search hint on) and the oracle over the given
    positions (one array per step, set before that step) and compares every
    step."""
    ctx = sidm.Context(n_ngb=n_ngb, box=p.box, estimator=int(overlap_table is not None),
                       search_hint=True)
    if overlap_table is not None:
        ctx.set_overlap_table(overlap_table)
    ctx.set_particles(positions[0], p.vel, p.ids, mass=p.mass)
    vel, h, dl = p.vel.copy(), np.zeros(p.n), np.full(p.n, np.inf)
    for k, (pos, act) in enumerate(zip(positions, masks)):
        if k > 0:
            ctx.set_positions(pos)
        o = oracle.step(pos, vel, p.mass, p.ids, act, bins, dt_max, n_ngb=n_ngb, box=p.box,
                        seed=seed, step=k, h_init=h, dtlim_init=dl,
                        overlap_table=overlap_table)
        g = _gpu_step(ctx, p, act, bins, dt_max, seed=seed)
        _compare(g, o, act, f"step {k}")
        vel, h, dl = o["vel"], o["h"], o["dtlim"]
    ctx.close()
    return o


def test_repeated_steps_of_a_halo_at_the_bench_neighbour_number():
    """N_ngb = 64 and the 512-particle window, as the benchmark runs: every
    step after the first starts from the last h of its active particles."""
    p = I.hernquist_halo(1 << 16, 21, ids="random")
    rng = np.random.default_rng(22)
    bins = rng.integers(0, 3, p.n).astype(np.int8)
    masks = [I.active_at_step(bins, s) for s in range(4)]
    o = _steps(p, [p.pos] * 4, masks, bins, 1.0, n_ngb=64)
    assert o["n_pairs"] > 10


@pytest.mark.parametrize("f", [0.3, 0.5, 0.9, 1.1, 2.0, 3.0])
def test_positions_rescaled_between_steps(f):
    """The halo contracted (f < 1: density x f^-3) or expanded (f > 1)
    about its centre after the first step.  At f = 0.3 the first radius
    holds ~37x the particles wanted, more than the gather list holds; at
    0.5 ~8x (kept); at 2 and 3 far fewer than K (the window takes over)."""
    p = I.hernquist_halo(20000, 23)
    pos2 = p.pos * f
    act = np.ones(p.n, np.uint8)
    bins = np.zeros(p.n, np.int8)
    _steps(p, [p.pos, pos2, pos2], [act, act, act], bins, 0.5)


def test_box_positions_shuffled_between_steps():
    """Every particle moved to another particle's place (periodic box): the
    last h says nothing about the new neighbourhood."""
    p = I.uniform_box(6000, 1.0, 1.0, 24, ids="random")
    rng = np.random.default_rng(25)
    dense = p.pos.copy()
    dense[: p.n // 2] *= 0.25          # half the particles crowded into a corner
    pos2 = dense[rng.permutation(p.n)]
    act = np.ones(p.n, np.uint8)
    _steps(p, [p.pos, pos2, p.pos], [act, act, act], np.zeros(p.n, np.int8), 0.05)


def test_overlap_estimator_repeated_steps():
    """Kernel-overlap estimator (Eq. 15): every particle is searched, each
    from its own last h after the first step."""
    p = I.hernquist_halo(12000, 26, ids="random")
    rng = np.random.default_rng(27)
    bins = rng.integers(0, 3, p.n).astype(np.int8)
    table = oracle.overlap_table(32, 128, kernel=0)
    masks = [I.active_at_step(bins, s) for s in range(3)]
    _steps(p, [p.pos, p.pos * 0.7, p.pos * 0.7], masks, bins, 2.0, overlap_table=table)


def test_hint_off_and_on_give_the_same_steps():
    """The plain form (no hint) and the hinted form step the same halo to
    bit-identical h, pairs and velocities."""
    p = I.hernquist_halo(30000, 28, ids="random")
    rng = np.random.default_rng(29)
    bins = rng.integers(0, 3, p.n).astype(np.int8)
    out = []
    for hint in (False, True):
        ctx = sidm.Context(n_ngb=64, box=0.0, search_hint=hint)
        ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
        res = []
        for s in range(4):
            ctx.step(1.0, I.active_at_step(bins, s), bins, seed=13)
            v, h = ctx.velocities()
            res.append((v.copy(), h.copy(), ctx.pairs()))
        ctx.close()
        out.append(res)
    for (v0, h0, (ab0, o0)), (v1, h1, (ab1, o1)) in zip(*out):
        assert np.array_equal(h0, h1)
        assert np.array_equal(ab0, ab1) and np.array_equal(o0, o1)
        assert np.array_equal(v0, v1)
