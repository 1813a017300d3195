"""Pins of the kinetic Boltzmann solver (Appendix B1), the second CPU
reference of the thermalisation test: what the equation and the scheme fix,
independent of the solver's own arithmetic."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.kinetic import KineticSolver

TAU = math.sqrt(3.0 * math.pi) / 4.0          # collision time for rho = sigma/m = v0 = 1


def _k4(ks, f):
    """<v^4> / <v^2>^2 (1 for one speed, 5/3 for Maxwell-Boltzmann)."""
    return (4.0 * ks.E ** 2 * f).sum() / (2.0 * ks.E * f).sum() ** 2 * f.sum()


def _loss_rate_of_mono_speed(ks, f):
    i, j = ks.pairs
    k0 = int(np.argmax(f))
    return 2.0 * f[k0] * ks.R[(i == k0) & (j == k0)][0]


@pytest.fixture(scope="module")
def const():
    return KineticSolver(1.0, lambda u: np.ones_like(u), e_max=5.0, n=81, n_delta=24)


def test_number_and_energy_are_kept(const):
    f0 = const.mono_speed(1.0)
    f = const.evolve(f0, 5.0 * TAU, TAU / 200)["final"]
    assert abs(const.number(f) - 1.0) < 1e-5
    assert abs(const.energy(f) - 0.5) < 1e-5


def test_out_scattering_rate_of_one_speed(const):
    """All particles at speed v0 with isotropic directions: the mean relative
    speed is 4 v0 / 3, so each particle leaves at rate rho (sigma/m) 4 v0 / 3."""
    f0 = const.mono_speed(1.0)
    assert abs(_loss_rate_of_mono_speed(const, f0) / (4.0 / 3.0) - 1.0) < 2e-3


def test_out_scattering_rate_with_a_velocity_dependent_cross_section():
    s0, w = 3.0, 1.0
    sig = lambda u: s0 / (1.0 + (u / w) ** 2) ** 2
    ks = KineticSolver(2.0, sig, e_max=5.0, n=81, n_delta=48)
    f0 = ks.mono_speed(1.0)
    # isotropic angle: u = sqrt(2 - 2c), c uniform on [-1, 1]
    want = 2.0 * integrate.quad(lambda c: 0.5 * sig(math.sqrt(2 - 2 * c)) * math.sqrt(2 - 2 * c),
                                -1.0, 1.0)[0]
    assert abs(_loss_rate_of_mono_speed(ks, f0) / want - 1.0) < 2e-3


def test_maxwell_boltzmann_is_nearly_stationary(const):
    fm = const.maxwell_boltzmann(1.0)
    d = const.dfdt(fm)
    i, j = const.pairs
    F = fm[i] * fm[j]
    scale = 2.0 * (F * const.R).sum()              # total loss rate of the density
    assert np.abs(d).sum() < 0.05 * scale


def test_relaxes_to_maxwell_boltzmann_and_converges_with_resolution(const):
    f0 = const.mono_speed(1.0)
    out = const.evolve(f0, 10.0 * TAU, TAU / 200, record=[TAU, 3 * TAU])
    assert _k4(const, out[TAU]) > 1.15 and _k4(const, out[3 * TAU]) > 1.4
    assert abs(_k4(const, out["final"]) - 5.0 / 3.0) < 0.01
    fine = KineticSolver(1.0, lambda u: np.ones_like(u), e_max=5.0, n=161, n_delta=24)
    o2 = fine.evolve(fine.mono_speed(1.0), 3.0 * TAU, TAU / 200, record=[TAU, 3 * TAU])
    for t in (TAU, 3 * TAU):
        assert abs(_k4(const, out[t]) - _k4(fine, o2[t])) < 0.006
