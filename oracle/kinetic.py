"""Kinetic Boltzmann solver for the thermalisation test -- TEST INFRASTRUCTURE.

A second CPU reference, independent of the N-body path: the homogeneous,
isotropic collisional Boltzmann equation for the energy distribution f(E, t)
with isotropic elastic scattering (Appendix B1, the reference solution of
the thermalisation test of Sec. 5.2).  Only ``tests/`` may import it.

Discretisation (Appendix B1):
  * energy nodes E_k = k dE, k = 0 .. n-1; f_k is the density per unit
    energy at E_k (sum_k f_k dE = 1 for a normalised distribution);
  * the angle delta between the incoming velocities is uniform in cos(delta),
    taken at the midpoints of n_delta bins;
  * for a bin pair i <= j and angle delta: the centre-of-momentum speed V,
    the relative speed u, and the outgoing energy E', uniform on
    [(V - u/2)^2 / 2, (V + u/2)^2 / 2] for isotropic scattering; I(E') is the
    antiderivative of its cumulative distribution;
  * events per unit time: rho (sigma(u)/m) u n_ij f_i f_j dE^2 dcos/2, with
    n_ij = 1/2 for i = j (an unordered pair of bins counts once);
  * each event puts one particle into the nodes around E' with the lever
    weights Lambda_k (so number and energy are kept), through the second
    difference of I, and the partner likewise at E_i + E_j - E' -- which has
    the same distribution, so both together give twice the forward term --
    and takes one particle out of bin i and one out of bin j.

The collision term is bilinear in f, so it is assembled once as a tensor
G[i, j, k] (gain at node k per unit f_i f_j) and a matrix R[i, j] (events
per unit f_i f_j dE^2, divided by dE: the loss of density at bins i and j);
time is advanced with the explicit midpoint rule.
"""
from __future__ import annotations

import math

import numpy as np


def _I(E, emin, emax):
    """Antiderivative of the CDF of a uniform distribution on [emin, emax]
    (0 below; (E - emin)^2 / (2 w) inside; w/2 + (E - emax) above)."""
    w = emax - emin
    inside = np.where(w > 0, (E - emin) ** 2 / (2.0 * np.where(w > 0, w, 1.0)), 0.0)
    above = 0.5 * w + (E - emax)
    return np.where(E <= emin, 0.0, np.where(E >= emax, above, inside))


class KineticSolver:
    """f(E, t) of a homogeneous box with isotropic elastic scattering at the
    rate rho (sigma(u)/m) u (sigma_over_m(u): a function of the relative
    speed, vectorised)."""

    def __init__(self, rho, sigma_over_m, e_max=5.0, n=80, n_delta=24):
        self.rho = float(rho)
        self.dE = e_max / (n - 1)
        self.E = np.arange(n) * self.dE
        dE = self.dE
        v = np.sqrt(2.0 * self.E)
        dc = 2.0 / n_delta
        cos_d = -1.0 + (np.arange(n_delta) + 0.5) * dc
        i, j = np.triu_indices(n)
        nij = np.where(i == j, 0.5, 1.0)
        vi, vj = v[i], v[j]
        # energy nodes -1 .. n for the second differences
        Eg = (np.arange(-1, n + 1) * dE)[None, :]
        G = np.zeros((i.size, n))
        R = np.zeros(i.size)
        for c in cos_d:
            V = 0.5 * np.sqrt(vi * vi + vj * vj + 2.0 * vi * vj * c)
            u = np.sqrt(np.maximum(vi * vi + vj * vj - 2.0 * vi * vj * c, 0.0))
            emin = 0.5 * (V - 0.5 * u) ** 2
            emax = 0.5 * (V + 0.5 * u) ** 2
            rate = self.rho * sigma_over_m(u) * u * nij * 0.5 * dc
            Ig = _I(Eg, emin[:, None], emax[:, None])
            d2 = Ig[:, 2:] - 2.0 * Ig[:, 1:-1] + Ig[:, :-2]
            # forward particle and partner (same distribution): 2 x lever gain
            G += (2.0 * rate)[:, None] * d2
            R += rate * dE
        self.n = n
        self.pairs = (i, j)
        self.G = G
        self.R = R

    def dfdt(self, f: np.ndarray) -> np.ndarray:
        i, j = self.pairs
        F = f[i] * f[j]
        gain = F @ self.G
        loss = np.zeros(self.n)
        np.add.at(loss, i, F * self.R)
        np.add.at(loss, j, F * self.R)
        return gain - loss

    def mono_speed(self, v0: float) -> np.ndarray:
        """All particles at speed v0 (E0 = v0^2 / 2 must be a node)."""
        k0 = int(round(0.5 * v0 * v0 / self.dE))
        if abs(k0 * self.dE - 0.5 * v0 * v0) > 1e-12 * self.dE * max(k0, 1):
            raise ValueError("E0 = v0^2 / 2 is not an energy node")
        f = np.zeros(self.n)
        f[k0] = 1.0 / self.dE
        return f

    def maxwell_boltzmann(self, v0: float) -> np.ndarray:
        """The MB energy density with <v^2> = v0^2 (kT = v0^2 / 3 per unit
        mass), f(E) ~ sqrt(E) exp(-E / kT), normalised on the nodes."""
        kt = v0 * v0 / 3.0
        f = np.sqrt(self.E) * np.exp(-self.E / kt)
        return f / (f.sum() * self.dE)

    def evolve(self, f0: np.ndarray, t_end: float, dt: float, record=None) -> dict:
        """Explicit midpoint rule; returns {t: f} at the requested times."""
        f = f0.astype(np.float64).copy()
        out = {}
        times = sorted(record or [])
        t, k = 0.0, 0
        steps = int(math.ceil(t_end / dt - 1e-9))
        for s in range(steps):
            while k < len(times) and times[k] <= t + 1e-12:
                out[times[k]] = f.copy()
                k += 1
            h = min(dt, t_end - t)
            mid = f + 0.5 * h * self.dfdt(f)
            f = f + h * self.dfdt(mid)
            t += h
        while k < len(times):
            out[times[k]] = f.copy()
            k += 1
        out["final"] = f
        return out

    # moments (per unit mass: E = v^2 / 2)
    def number(self, f):
        return float(f.sum() * self.dE)

    def energy(self, f):
        return float((self.E * f).sum() * self.dE)

    def mean_speed(self, f):
        return float((np.sqrt(2.0 * self.E) * f).sum() * self.dE / self.number(f))

    def speed_variance(self, f):
        """var|v| = <v^2> - <v>^2."""
        n = self.number(f)
        return 2.0 * self.energy(f) / n - self.mean_speed(f) ** 2
