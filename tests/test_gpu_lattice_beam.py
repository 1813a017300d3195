"""Beam through a lattice of targets at rest (Sec. 5.1), scaled down.

Targets sit on a 48^3 lattice of density 1; 3000 beam particles of the same
mass move with v = (1, 0, 0).  Target-target and beam-beam pairs have zero
relative speed and cannot scatter, so an unscattered beam particle meets
only targets and leaves the beam at the rate Gamma = rho (sigma/m) v = 1.
The unscattered fraction must follow exp(-Gamma t), and every step must
conserve energy and momentum to round-off.  The step runs on fixed
positions: only the scattering substep is tested.
"""
import math

import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu

N_SIDE, N_BEAM, DT, STEPS = 48, 3000, 0.04, 30


def test_beam_decays_at_the_scattering_rate():
    p = I.lattice_beam(N_SIDE, N_BEAM, seed=11)
    nt = p.meta["n_target"]
    ctx = sidm.Context(n_ngb=32, box=p.box)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    bins = np.zeros(p.n, np.int8)
    beam_v = p.vel[nt:].copy()
    surv = []
    for s in range(STEPS):
        st = ctx.step(DT, None, bins, sigma0=1.0, seed=3)
        assert st["return"] >= 0
        assert abs(st["e_after"] - st["e_before"]) <= 1e-12 * st["e_before"]
        for k in range(3):
            assert abs(st["p_after"][k] - st["p_before"][k]) <= 1e-12 * N_BEAM * p.mass[0]
        v, _ = ctx.velocities()
        # a beam particle is unscattered while its velocity is bit-identical
        surv.append(int(np.all(v[nt:] == beam_v, axis=1).sum()))
    ctx.close()
    t = DT * np.arange(1, STEPS + 1)
    f = np.array(surv) / N_BEAM
    assert np.all(np.diff(surv) <= 0)            # a scattered particle never returns
    # least-squares decay rate of log f(t) through the origin
    gamma = -np.sum(t * np.log(f)) / np.sum(t * t)
    assert abs(gamma - 1.0) < 0.08, gamma
    # the final count against the binomial spread around exp(-Gamma T)
    q = math.exp(-t[-1])
    sd = math.sqrt(N_BEAM * q * (1 - q))
    assert abs(surv[-1] - N_BEAM * q) < 5 * sd, (surv[-1], N_BEAM * q, sd)
