"""Thermalisation in a periodic box (the paper's test of this path, Sec. 5.2).

Particles start with one speed v0 and isotropic directions; elastic SIDM
scatters drive the speeds to the Maxwell-Boltzmann distribution of the same
mean energy, f(v) = 4 pi v^2 (3 / (2 pi v0^2))^(3/2) exp(-3 v^2 / (2 v0^2)),
on the collision time tau = sqrt(3 pi) / (4 v0 (sigma/m) rho).  Positions
drift x += v dt between scattering steps (no gravity).  Energy and momentum
are conserved to round-off throughout.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _mb_cdf(v, v0):
    # CDF of the Maxwell-Boltzmann speed distribution with <v^2> = v0^2
    a = v0 / math.sqrt(3.0)
    x = v / (math.sqrt(2.0) * a)
    return [math.erf(t) - math.sqrt(2.0 / math.pi) * (vv / a) * math.exp(-t * t)
            for t, vv in zip(x, v)]


@pytest.mark.parametrize("sigma_kind", [sidm.SIGMA_CONST, sidm.SIGMA_YUKAWA])
def test_mono_speed_box_relaxes_to_maxwell_boltzmann(sigma_kind):
    n, v0, L = 10000, 1.0, 1.0
    p = I.mono_speed_box(n, L, v0, seed=4)
    rho = 1.0
    # Yukawa-like: sigma0/m / (1 + (v/w)^2)^2 with w = v0; the collision time
    # uses sigma/m at the mean MB relative speed 4 v0 / sqrt(3 pi)
    w = v0
    vrel = 4.0 * v0 / math.sqrt(3.0 * math.pi)
    s_eff = 1.0 / (1.0 + (vrel / w) ** 2) ** 2 if sigma_kind == sidm.SIGMA_YUKAWA else 1.0
    sigma0 = 1.0 / s_eff
    tau = math.sqrt(3.0 * math.pi) / (4.0 * v0 * 1.0 * rho)
    dt = 0.05 * tau
    ctx = sidm.Context(n_ngb=32, box=L)
    pos, vel = p.pos.copy(), p.vel.copy()
    ctx.set_particles(pos, vel, p.ids, mass=p.mass)
    e0 = 0.5 * (p.mass * (vel ** 2).sum(1)).sum()
    p0 = (p.mass[:, None] * vel).sum(0)
    ks = {}
    steps = int(round(8.0 * tau / dt))
    for k in range(steps):
        ctx.step(dt, None, None, sigma0=sigma0, sigma_kind=sigma_kind, w=w, seed=11, stats=False)
        vel, _ = ctx.velocities()
        pos = np.mod(pos + vel * dt, L)
        pos[pos >= L] = 0.0
        ctx.set_particles(pos, vel, p.ids, mass=p.mass)
        ctx.step_counter = k + 1
        t = (k + 1) * dt / tau
        if abs(t - 1.0) < 1e-9 or k + 1 == steps:
            sp = np.linalg.norm(vel, axis=1)
            r = stats.kstest(sp, lambda x: np.array(_mb_cdf(np.atleast_1d(x), v0)))
            ks[round(t, 3)] = (r.pvalue, r.statistic)
    ctx.close()
    e1 = 0.5 * (p.mass * (vel ** 2).sum(1)).sum()
    p1 = (p.mass[:, None] * vel).sum(0)
    assert abs(e1 - e0) <= 1e-11 * e0
    assert np.max(np.abs(p1 - p0)) <= 1e-13 * (p.mass[:, None] * np.abs(vel)).sum()
    sp = np.linalg.norm(vel, axis=1)
    assert abs(np.mean(sp ** 2) / v0 ** 2 - 1.0) < 1e-9
    p_end, d_end = ks[max(ks)]
    p_one, d_one = ks[1.0]
    if sigma_kind == sidm.SIGMA_CONST:
        # relaxed after 8 collision times: the speeds follow MB
        assert p_end > 1e-3
    # approaching MB: the KS distance shrinks well below its value at 1 tau
    # (the Yukawa-like law scatters the fast tail ~100x less, so it relaxes
    # more slowly; the paper compares that case with a kinetic solver)
    assert d_end < d_one / 3.0


def _k4(v):
    """<v^4> / <v^2>^2 of the speeds: 1 for one speed, 5/3 for MB."""
    s2 = (v * v).sum(1)
    return float(np.mean(s2 * s2) / np.mean(s2) ** 2)


@pytest.mark.parametrize("sigma_kind", [sidm.SIGMA_CONST, sidm.SIGMA_YUKAWA])
def test_relaxation_rate_follows_the_kinetic_solver(sigma_kind):
    """The relaxation itself, not only its end state: the fourth speed moment
    K = <v^4> / <v^2>^2 rises from 1 (one speed) towards 5/3 (MB) on the
    collision time, and the N-body path follows the kinetic Boltzmann
    solution of the same box (Appendix B1; oracle.kinetic) at 1, 2 and 3
    collision times within 0.03 in K.  That bound covers the sampling noise
    of K with 2^17 particles (about 0.008), the first-order time error of
    steps of tau/20 (about 0.01) and the solver's grid (below 0.005); a rate
    off by 25 % moves K(tau) by about 0.05."""
    from oracle.kinetic import KineticSolver
    n, v0, L = 1 << 17, 1.0, 1.0
    p = I.mono_speed_box(n, L, v0, seed=9)
    rho = 1.0
    tau = math.sqrt(3.0 * math.pi) / (4.0 * v0 * 1.0 * rho)
    w = v0
    if sigma_kind == sidm.SIGMA_YUKAWA:
        vrel = 4.0 * v0 / math.sqrt(3.0 * math.pi)
        sigma0 = (1.0 + (vrel / w) ** 2) ** 2
        sig = lambda u: sigma0 / (1.0 + (u / w) ** 2) ** 2
    else:
        sigma0 = 1.0
        sig = lambda u: np.full_like(u, sigma0)
    dt = tau / 20.0
    ctx = sidm.Context(n_ngb=32, box=L, n_max=n)
    pos, vel = p.pos.copy(), p.vel.copy()
    ctx.set_particles(pos, vel, p.ids, mass=p.mass)
    k_gpu = {}
    for k in range(60):
        ctx.step(dt, None, None, sigma0=sigma0, sigma_kind=sigma_kind, w=w, seed=21, stats=False)
        vel, _ = ctx.velocities()
        if (k + 1) % 20 == 0:
            k_gpu[(k + 1) // 20] = _k4(vel)
        pos = np.mod(pos + vel * dt, L)
        pos[pos >= L] = 0.0
        ctx.set_positions(pos)
    ctx.close()
    ks = KineticSolver(rho, sig, e_max=5.0, n=81, n_delta=24)
    out = ks.evolve(ks.mono_speed(v0), 3.0 * tau, tau / 200, record=[tau, 2 * tau, 3 * tau])
    for m in (1, 2, 3):
        f = out[m * tau]
        k_kin = (4.0 * ks.E ** 2 * f).sum() / (2.0 * ks.E * f).sum() ** 2 * f.sum()
        assert abs(k_gpu[m] - k_kin) <= 0.03, (sigma_kind, m, k_gpu[m], k_kin)
    assert k_gpu[3] - 1.0 > 0.5 * (2.0 / 3.0)       # past half of the relaxation


@pytest.mark.parametrize("c_sidm", [0.1, 1.0, 5.0])
def test_timestep_from_the_criterion_alone(c_sidm):
    """The paper's C_SIDM scan of this test (Sec. 5.2): no external maximum
    timestep, so the Eq. 18 limits alone set dt (here one global
    power-of-two step, the finest any particle needs).  With N_ngb = 32 the
    criterion's step is about 3.9 C_SIDM collision times, so C_SIDM = 5
    takes steps of 16 collision times; a pair scatters at most once per step,
    so such steps scatter less than their length suggests, and the run takes
    at least three of them.  The speeds end at the MB spread (and, for
    C_SIDM <= 1, pass a KS test against MB), with energy and momentum
    conserved to round-off."""
    n, v0, L = 10000, 1.0, 1.0
    p = I.mono_speed_box(n, L, v0, seed=7)
    tau = math.sqrt(3.0 * math.pi) / (4.0 * v0 * 1.0 * 1.0)
    dt_max = 64.0 * tau
    ctx = sidm.Context(n_ngb=32, box=L, c_sidm=c_sidm, pair_capacity=60 * n)
    pos, vel = p.pos.copy(), p.vel.copy()
    ctx.set_particles(pos, vel, p.ids, mass=p.mass)
    e0 = 0.5 * (p.mass * (vel ** 2).sum(1)).sum()
    p0 = (p.mass[:, None] * vel).sum(0)
    b = 12                               # bootstrap step (dt = dt_max / 4096) gives the limits
    t, steps, p_ge_1 = 0.0, 0, 0
    while t < 8.0 * tau or steps < 4:   # the bootstrap step and at least 3 more
        dt = math.ldexp(dt_max, -b)
        st = ctx.step(dt_max, None, np.full(n, b, np.int8), seed=13, stats=True)
        p_ge_1 += st["n_p_ge_1"]
        vel, _ = ctx.velocities()
        lim = ctx.timestep_limits()          # Eq. 18, from this step's velocities
        pos = np.mod(pos + vel * dt, L)
        pos[pos >= L] = 0.0
        ctx.set_particles(pos, vel, p.ids, mass=p.mass)
        steps += 1
        ctx.step_counter = steps
        t += dt
        # next step: the finest bin b with dt_max 2^-b below every limit
        assert np.all(np.isfinite(lim)) and lim.min() > 0.0
        need = np.ceil(np.log2(dt_max / lim.min()))
        b = int(max(0, need if math.ldexp(dt_max, -int(need)) < lim.min() else need + 1))
    ctx.close()
    e1 = 0.5 * (p.mass * (vel ** 2).sum(1)).sum()
    p1 = (p.mass[:, None] * vel).sum(0)
    assert abs(e1 - e0) <= 1e-11 * e0
    assert np.max(np.abs(p1 - p0)) <= 1e-13 * (p.mass[:, None] * np.abs(vel)).sum()
    sp = np.linalg.norm(vel, axis=1)
    ks = stats.kstest(sp, lambda x: np.array(_mb_cdf(np.atleast_1d(x), v0)))
    # MB with <v^2> = v0^2 has var|v| = v0^2 (1 - 8 / (3 pi)); the mono-speed start has 0
    var_mb = v0 ** 2 * (1.0 - 8.0 / (3.0 * math.pi))
    assert abs(np.var(sp) / var_mb - 1.0) < 0.05, (c_sidm, steps, np.var(sp) / var_mb)
    assert ks.statistic < 0.05, (c_sidm, steps, ks)
    if c_sidm <= 1.0:
        # up to a step of about 4 collision times the speeds pass as MB
        assert ks.pvalue > 1e-3, (c_sidm, steps, ks)
    # the criterion's step is about 3.9 C_SIDM collision times (Sec. 4.4 with
    # N_ngb = 32 and the mono-speed v_max = 2 v0), rounded down to a power of two
    assert steps <= int(8.0 / (0.1 * c_sidm)) + 4
