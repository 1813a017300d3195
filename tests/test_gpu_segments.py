"""Sub-ranges of a loaded context (sidm_write_particles, sidm_read_particles,
sidm_set_count): a halo written into a segment of a context that holds
other haloes steps exactly as it does alone, and writing, reading or
dropping one segment leaves the others as they were."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _alone(p, bins, dt, steps, seed):
    c = sidm.Context(n_ngb=32)
    c.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    for s in range(steps):
        c.step_counter = s
        c.step(dt, I.active_at_step(bins, s), bins, seed=seed, stats=False)
    v, h = c.velocities()
    c.close()
    return v, h


def test_segment_written_into_a_resident_context_steps_as_alone():
    a = I.hernquist_halo(6000, 21)
    b = I.hernquist_halo(9000, 22)
    c2 = I.nfw_halo(4000, 23)
    ba, dta = I.timestep_bins(a, I.hernquist_density, 1.0, 32)
    bb, dtb = I.timestep_bins(b, I.hernquist_density, 2.0, 32)
    bc, dtc = I.timestep_bins(c2, I.nfw_density, 0.5, 32)
    ctx = sidm.Context(n_ngb=32, n_max=20000)
    z = np.zeros((0, 3))
    ctx.set_particles(z, z, np.zeros(0, np.uint32), mass_scalar=1.0)
    ctx.write_particles(0, a.pos, a.vel, a.ids, mass=a.mass)
    ctx.write_particles(a.n, b.pos, b.vel, b.ids, mass=b.mass)
    assert ctx.n == a.n + b.n
    off = [0, a.n, a.n + b.n]
    ctx.set_haloes(off)
    bins = np.concatenate([ba, bb])

    def params(s, dts, seeds):
        return [sidm.HaloParams(dt, sidm.SigmaModel(0, 1.0, 1.0), sd, s)
                for dt, sd in zip(dts, seeds)]

    for s in range(3):
        act = np.concatenate([I.active_at_step(ba, s), I.active_at_step(bb, s)])
        sidm.sidm_step_haloes(ctx.handle, act, bins, params(s, [dta, dtb], [1, 2]), None)
    va = ctx.read_velocities(0, a.n)
    assert np.array_equal(va, _alone(a, ba, dta, 3, 1)[0])
    # replace halo b by c2 (smaller: the loaded count stays, the tail becomes a hole)
    ctx.write_particles(a.n, c2.pos, c2.vel, c2.ids, mass=c2.mass)
    off = [0, a.n, a.n + c2.n, a.n + b.n]
    ctx.set_haloes(off)
    hole = np.zeros(b.n - c2.n, np.uint8)
    bins = np.concatenate([ba, bc, np.zeros(b.n - c2.n, np.int8)])
    for s in range(3, 6):
        act = np.concatenate([I.active_at_step(ba, s), I.active_at_step(bc, s - 3), hole])
        prm = params(s, [dta, dtc, 1.0], [1, 3, 0])
        prm[1].step = s - 3
        sidm.sidm_step_haloes(ctx.handle, act, bins, prm, None)
    assert np.array_equal(ctx.read_velocities(0, a.n), _alone(a, ba, dta, 6, 1)[0])
    vc = ctx.read_velocities(a.n, c2.n)
    assert np.array_equal(vc, _alone(c2, bc, dtc, 3, 3)[0])
    # drop the hole at the end; halo a and c2 are untouched
    ctx.set_count(a.n + c2.n)
    ctx.set_haloes([0, a.n, a.n + c2.n])
    assert np.array_equal(ctx.read_velocities(a.n, c2.n), vc)
    with pytest.raises(sidm.SidmError):
        ctx.write_particles(20000 - 10, a.pos[:11], a.vel[:11], a.ids[:11])   # past capacity
    with pytest.raises(sidm.SidmError):
        ctx.write_particles(ctx.n + 1, a.pos[:2], a.vel[:2], a.ids[:2])        # a gap
    ctx.close()


def test_a_halo_moved_into_a_hole_steps_as_before():
    """sidm_move_particles: a halo moved as a whole (to close a hole left by
    a retired one) continues exactly as if it had stayed."""
    a = I.hernquist_halo(5000, 31)
    gone = I.hernquist_halo(7000, 32)
    b = I.nfw_halo(3000, 33)
    ba, dta = I.timestep_bins(a, I.hernquist_density, 1.0, 32)
    bg, dtg = I.timestep_bins(gone, I.hernquist_density, 1.0, 32)
    bb, dtb = I.timestep_bins(b, I.nfw_density, 2.0, 32)
    ctx = sidm.Context(n_ngb=32, n_max=20000)
    z = np.zeros((0, 3))
    ctx.set_particles(z, z, np.zeros(0, np.uint32), mass_scalar=1.0)
    for off, h in ((0, a), (a.n, gone), (a.n + gone.n, b)):
        ctx.write_particles(off, h.pos, h.vel, h.ids, mass=h.mass)
    ctx.set_haloes([0, a.n, a.n + gone.n, a.n + gone.n + b.n])

    def params(s, sb, three=True):
        p = [sidm.HaloParams(dta, sidm.SigmaModel(0, 1.0, 1.0), 1, s)]
        if three:
            p.append(sidm.HaloParams(dtg, sidm.SigmaModel(0, 1.0, 1.0), 2, s))
        p.append(sidm.HaloParams(dtb, sidm.SigmaModel(0, 1.0, 1.0), 3, sb))
        return p

    for s in range(3):
        act = np.concatenate([I.active_at_step(ba, s), I.active_at_step(bg, s),
                              I.active_at_step(bb, s)])
        sidm.sidm_step_haloes(ctx.handle, act, np.concatenate([ba, bg, bb]), params(s, s), None)
    # the middle halo retires; b moves down into its place and the tail goes
    ctx.move_particles(a.n + gone.n, a.n, b.n)
    ctx.set_count(a.n + b.n)
    ctx.set_haloes([0, a.n, a.n + b.n])
    for s in range(3, 6):
        act = np.concatenate([I.active_at_step(ba, s), I.active_at_step(bb, s)])
        sidm.sidm_step_haloes(ctx.handle, act, np.concatenate([ba, bb]), params(s, s, False),
                              None)
    va = ctx.read_velocities(0, a.n)
    vb = ctx.read_velocities(a.n, b.n)
    ctx.close()
    assert np.array_equal(va, _alone(a, ba, dta, 6, 1)[0])
    assert np.array_equal(vb, _alone(b, bb, dtb, 6, 3)[0])


@pytest.mark.parametrize("src,dst,count", [(100, 50, 1000), (50, 100, 1000), (0, 3, 997),
                                           (2000, 0, 700), (10, 10, 5)])
def test_move_particles_with_overlapping_ranges(src, dst, count):
    p = I.uniform_box(3000, 1.0, 1.0, 41)
    ctx = sidm.Context(n_max=3000)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.move_particles(src, dst, count)
    v = ctx.read_velocities(0, p.n)
    want = p.vel.copy()
    want[dst:dst + count] = p.vel[src:src + count]
    assert np.array_equal(v, want)
    with pytest.raises(sidm.SidmError):
        ctx.move_particles(2500, 0, 600)            # source past the loaded count
    ctx.close()
