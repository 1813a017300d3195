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
