"""sidm_get_changed: the particles whose velocities the last step changed,
each once, with their new velocities.  A host copy of the velocities kept
up to date from these deltas alone must equal the full read-back."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def test_changed_set_is_the_particles_of_the_accepted_pairs():
    p = I.hernquist_halo(20000, 41, ids="random")
    bins = np.random.default_rng(42).integers(0, 3, p.n).astype(np.int8)
    where = {int(i): k for k, i in enumerate(p.ids)}
    ctx = sidm.Context(n_ngb=32, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    idx, v = ctx.changed()
    assert idx.size == 0                       # no step yet
    host = p.vel.copy()
    total = 0
    for k in range(6):
        before = ctx.velocities()[0]
        ctx.step(2.0, I.active_at_step(bins, k), bins, seed=43, stats=False)
        after = ctx.velocities()[0]
        idx, v = ctx.changed()
        assert np.unique(idx).size == idx.size
        ab, _ = ctx.pairs()
        kicked = {where[int(i)] for i in ab.ravel()}
        assert set(idx.tolist()) == kicked, k
        assert np.array_equal(v, after[idx])
        moved = np.nonzero(np.any(after != before, axis=1))[0]
        assert set(moved.tolist()) <= kicked
        host[idx] = v
        assert np.array_equal(host, after), k
        total += idx.size
    assert total > 500
    # a new particle set starts with nothing changed
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    assert ctx.changed()[0].size == 0
    ctx.close()


def test_short_output_gets_the_full_count():
    p = I.uniform_box(4000, 1.0, 1.0, 44)
    ctx = sidm.Context(box=1.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.step(0.2, None, np.zeros(p.n, np.int8), seed=45, stats=False)
    full_idx, full_v = ctx.changed()
    assert full_idx.size > 10
    idx = np.full(5, -1, np.int32)
    vel = np.zeros((5, 3))
    n = sidm.sidm_get_changed(ctx.handle, idx, vel)
    assert n == full_idx.size
    assert set(idx.tolist()) <= set(full_idx.tolist())
    after = ctx.velocities()[0]
    assert np.array_equal(vel, after[idx])
    ctx.close()


def test_update_velocities_keeps_a_host_copy_current():
    p = I.hernquist_halo(15000, 46, ids="random")
    bins = np.random.default_rng(47).integers(0, 3, p.n).astype(np.int8)
    ctx = sidm.Context(n_ngb=32, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    host = p.vel.copy()
    sidm.sidm_update_velocities(ctx.handle, host)       # no step yet: untouched
    assert np.array_equal(host, p.vel)
    for k in range(5):
        ctx.step(2.0, I.active_at_step(bins, k), bins, seed=48, stats=False)
        sidm.sidm_update_velocities(ctx.handle, host)
        assert np.array_equal(host, ctx.velocities()[0]), k
    with pytest.raises(sidm.SidmError):
        sidm.sidm_update_velocities(ctx.handle, host.astype(np.float32))
    ctx.close()


def test_update_velocities_into_pinned_memory_writes_from_the_device():
    """A pinned host array (device-addressable) takes the changed particles'
    velocities straight from the device: it stays equal to the full
    read-back, and entries of particles the step did not change keep
    whatever they held."""
    torch = pytest.importorskip("torch")
    p = I.hernquist_halo(15000, 49, ids="random")
    bins = np.random.default_rng(50).integers(0, 3, p.n).astype(np.int8)
    ctx = sidm.Context(n_ngb=32, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    host = torch.from_numpy(p.vel.copy()).pin_memory().numpy()
    pageable = p.vel.copy()
    marked = torch.full((p.n, 3), np.nan, dtype=torch.float64).pin_memory().numpy()
    # the same, 8 bytes past a 16-byte boundary (one store per component)
    shifted = torch.from_numpy(np.concatenate([[0.0], p.vel.ravel()])).pin_memory().numpy()
    shifted = shifted[1:].reshape(p.n, 3)
    assert shifted.ctypes.data % 16 == 8
    launches = ctx.kernel_launches
    sidm.sidm_update_velocities(ctx.handle, host)       # no step yet: untouched
    assert np.array_equal(host, p.vel)
    assert ctx.kernel_launches == launches
    for k in range(5):
        ctx.step(2.0, I.active_at_step(bins, k), bins, seed=51, stats=False)
        before = ctx.kernel_launches
        sidm.sidm_update_velocities(ctx.handle, host)
        assert ctx.kernel_launches == before + 1       # the direct write, no staging
        sidm.sidm_update_velocities(ctx.handle, pageable)
        sidm.sidm_update_velocities(ctx.handle, marked)
        sidm.sidm_update_velocities(ctx.handle, shifted)
        after = ctx.velocities()[0]
        assert np.array_equal(host, after), k
        assert np.array_equal(shifted, after), k
        assert np.array_equal(pageable, after), k
        idx, v = ctx.changed()
        hit = np.zeros(p.n, bool)
        hit[idx] = True
        assert np.array_equal(marked[hit], after[hit])
        assert np.isnan(marked[~hit]).all()
        marked[:] = np.nan
    ctx.close()


def test_velocity_mirror_is_kept_current_by_the_kicks():
    """sidm_set_velocity_mirror: a pinned host array into which the step's
    kicks write each changed particle's final velocity.  After every step
    (and a wait for the stream) it equals the full read-back; only the
    particles the step changed are written; the velocities are bit for bit
    those of a context without the mirror (multiple scatters per particle
    at dt_max = 2); a mirror shorter than the particle set stops the step,
    autotuning leaves it alone, and pageable memory is refused."""
    torch = pytest.importorskip("torch")
    p = I.hernquist_halo(20000, 52, ids="random")
    bins = np.random.default_rng(53).integers(0, 3, p.n).astype(np.int8)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    ref = sidm.Context(n_ngb=32, use_graph=True)
    ref.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx = sidm.Context(n_ngb=32, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    mirror = pin(p.vel.copy())
    ctx.set_velocity_mirror(mirror)
    multi = 0
    for k in range(6):
        act = I.active_at_step(bins, k)
        ref.step(2.0, act, bins, seed=54, stats=False)
        st = ctx.step(2.0, act, bins, seed=54)
        multi = max(multi, st["max_multiplicity"])
        ctx.sync()
        after = ctx.velocities()[0]
        assert np.array_equal(after, ref.velocities()[0]), k
        assert np.array_equal(mirror, after), k
    assert multi >= 3
    # only the changed particles are written
    marked = pin(np.full((p.n, 3), np.nan))
    ctx.set_velocity_mirror(marked)
    ctx.step(2.0, I.active_at_step(bins, 6), bins, seed=54, stats=False)
    ctx.sync()
    after = ctx.velocities()[0]
    idx, _ = ctx.changed()
    hit = np.zeros(p.n, bool)
    hit[idx] = True
    assert hit.sum() > 100
    assert np.array_equal(marked[hit], after[hit])
    assert np.isnan(marked[~hit]).all()
    # trial steps of the autotuner leave the mirror alone
    marked[:] = np.nan
    ctx.autotune([sidm.HaloParams(2.0, sidm.SigmaModel(0, 1.0, 1.0), 54, ctx.step_counter)],
                 I.active_at_step(bins, 7), bins, reps=1)
    assert np.isnan(marked).all()
    # too short for the particle set: the step is refused
    ctx.set_velocity_mirror(pin(np.zeros((p.n - 1, 3))))
    with pytest.raises(sidm.SidmError):
        ctx.step(2.0, I.active_at_step(bins, 7), bins, seed=54, stats=False)
    ctx.set_velocity_mirror(None)
    ctx.step(2.0, I.active_at_step(bins, 7), bins, seed=54, stats=False)
    with pytest.raises(sidm.SidmError):
        ctx.set_velocity_mirror(np.zeros((p.n, 3)))   # pageable
    ctx.close()
    ref.close()
