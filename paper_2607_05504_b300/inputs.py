"""Seeded synthetic inputs for the SIDM scattering step.

This module only *generates inputs*: particle positions, velocities, masses,
ids, power-of-two timestep bins and active masks.  It holds none of the
scattering method's arithmetic (no neighbour search, kernel, probability,
random draw or kick); both the CUDA path and the CPU oracle consume what it
produces.  Every generator is deterministic in its ``seed`` (numpy PCG64).

Workloads (the paper runs its own tests on a uniform box, Sec. 5.2, and on
isolated haloes, Sec. 5.3; no dataset is involved):

* ``uniform_box``   periodic cube, uniform positions, Maxwellian velocities.
* ``hernquist_halo`` isolated Hernquist (1990) sphere, G = M = a = 1,
                     velocities from its closed-form ergodic distribution
                     function (the Eddington inversion of the profile).
* ``nfw_halo``       isolated NFW sphere truncated at ``c`` scale radii,
                     velocities from a numerical Eddington inversion.
* ``timestep_bins``  power-of-two bins from an analytic local collision-time
                     estimate, with ``dt_max`` chosen for a target mean
                     active fraction (individual timesteps, Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Particles:
    pos: np.ndarray          # (n, 3) float64, row-major
    vel: np.ndarray          # (n, 3) float64
    mass: np.ndarray         # (n,)  float64
    ids: np.ndarray          # (n,)  uint32, unique
    box: float = 0.0         # > 0: periodic cube side; 0: open boundaries
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def copy(self) -> "Particles":
        return Particles(self.pos.copy(), self.vel.copy(), self.mass.copy(),
                         self.ids.copy(), self.box, dict(self.meta))


def _ids(rng: np.random.Generator, n: int, kind: str) -> np.ndarray:
    if kind == "arange":
        return np.arange(n, dtype=np.uint32)
    if kind == "random":
        # unique ids spread over the whole 32-bit range (exercises min/max id
        # ordering independently of storage order)
        ids = rng.choice(np.uint64(2**32 - 1), size=n, replace=False)
        return ids.astype(np.uint32)
    raise ValueError(kind)


def uniform_box(n: int, box: float = 1.0, sigma_v: float = 1.0, seed: int = 0,
                mass_total: float | None = None, ids: str = "arange") -> Particles:
    """Uniform random positions in [0, box)^3, Gaussian velocity components.

    ``mass_total`` defaults to box**3 (mean density 1)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * box
    # guard against the rare value that rounds up to exactly ``box``
    pos[pos >= box] = 0.0
    vel = rng.standard_normal((n, 3)) * sigma_v
    mt = box ** 3 if mass_total is None else mass_total
    mass = np.full(n, mt / n)
    return Particles(pos, vel, mass, _ids(rng, n, ids), float(box),
                     {"kind": "box", "sigma_v": sigma_v, "rho": mt / box ** 3})


def mono_speed_box(n: int, box: float = 1.0, v0: float = 1.0, seed: int = 0,
                   mass_total: float | None = None) -> Particles:
    """Thermalisation set-up (Sec. 5.2): every particle has speed v0 and an
    isotropic direction."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * box
    pos[pos >= box] = 0.0
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    vel = d * v0
    mt = box ** 3 if mass_total is None else mass_total
    mass = np.full(n, mt / n)
    return Particles(pos, vel, mass, _ids(rng, n, "arange"), float(box),
                     {"kind": "mono", "v0": v0, "rho": mt / box ** 3})


def lattice_beam(n_side: int, n_beam: int, box: float = 1.0, v0: float = 1.0,
                 seed: int = 0) -> Particles:
    """Beam-through-lattice set-up (Sec. 5.1): n_side^3 targets at rest on a
    cubic lattice of total mass box^3 (density 1), and n_beam particles of the
    same mass at uniform random positions, all moving with velocity
    (v0, 0, 0).  The targets come first."""
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) + 0.5) * (box / n_side)
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    tgt = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    beam = rng.random((n_beam, 3)) * box
    beam[beam >= box] = 0.0
    pos = np.concatenate([tgt, beam])
    vel = np.zeros_like(pos)
    vel[tgt.shape[0]:, 0] = v0
    n = pos.shape[0]
    m = box ** 3 / tgt.shape[0]
    return Particles(pos, vel, np.full(n, m), _ids(rng, n, "random"), float(box),
                     {"kind": "lattice_beam", "n_target": tgt.shape[0], "v0": v0, "rho": 1.0})


# ---------------------------------------------------------------- haloes ---

def _isotropic(rng: np.random.Generator, r: np.ndarray) -> np.ndarray:
    u = rng.random(r.shape[0]) * 2.0 - 1.0
    phi = rng.random(r.shape[0]) * 2.0 * math.pi
    s = np.sqrt(1.0 - u * u)
    return np.stack([s * np.cos(phi), s * np.sin(phi), u], axis=1) * r[:, None]


def hernquist_df(E: np.ndarray) -> np.ndarray:
    """Hernquist (1990, eq. 17) ergodic distribution function for G = M = a = 1
    as a function of the relative energy E = psi - v^2/2 in (0, 1)."""
    q = np.sqrt(np.clip(E, 0.0, 1.0 - 1e-15))
    q2 = q * q
    br = 3.0 * np.arcsin(q) + q * np.sqrt(1.0 - q2) * (1.0 - 2.0 * q2) * (8.0 * q2 * q2 - 8.0 * q2 - 3.0)
    return br / (8.0 * math.sqrt(2.0) * math.pi ** 3 * (1.0 - q2) ** 2.5)


def _sample_speeds(rng, psi: np.ndarray, df, psi0: float) -> np.ndarray:
    """Rejection-sample speeds v in [0, sqrt(2 psi)] with density
    v^2 f(psi - v^2/2), per particle.  The envelope max_y y^2 f(psi(1-y^2))
    is tabulated once on a log grid of psi0 - psi (psi0 = psi at the centre,
    where the distribution function diverges) and taken, with a margin, as
    the larger of the two bracketing table values."""
    n = psi.shape[0]
    vesc = np.sqrt(2.0 * psi)
    y = np.linspace(0.0, 1.0, 193)[1:][None, :]
    d = np.maximum(psi0 - psi, 1e-300)
    dg = np.geomspace(d.min() * 0.999, d.max() * 1.001, 4096)
    pg = psi0 - dg
    tab = np.empty(pg.shape[0])
    for s in range(0, pg.shape[0], 256):
        ps = pg[s:s + 256, None]
        tab[s:s + 256] = (y * y * df(ps * (1.0 - y * y))).max(axis=1)
    idx = np.clip(np.searchsorted(dg, d), 1, dg.shape[0] - 1)
    gmax = 1.5 * np.maximum(tab[idx - 1], tab[idx])
    out = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        y = rng.random(todo.size)
        g = y * y * df(psi[todo] * (1.0 - y * y))
        ok = rng.random(todo.size) * gmax[todo] < g
        out[todo[ok]] = y[ok]
        todo = todo[~ok]
    return out * vesc


def hernquist_halo(n: int, seed: int = 1, r_trunc: float = 100.0,
                   ids: str = "arange") -> Particles:
    """Isolated Hernquist sphere, G = M = a = 1, radii from the inverse of
    M(<r) = r^2/(1+r)^2 restricted to r <= r_trunc; each particle carries
    mass M(<r_trunc)/n; velocities from the untruncated closed-form DF."""
    rng = np.random.default_rng(seed)
    xmax = (r_trunc / (1.0 + r_trunc)) ** 2
    X = rng.random(n) * xmax
    sx = np.sqrt(X)
    r = sx / (1.0 - sx)
    pos = _isotropic(rng, r)
    psi = 1.0 / (1.0 + r)
    v = _sample_speeds(rng, psi, hernquist_df, 1.0)
    vel = _isotropic(rng, v)
    mass = np.full(n, xmax / n)
    return Particles(pos, vel, mass, _ids(rng, n, ids), 0.0,
                     {"kind": "hernquist", "r_trunc": r_trunc})


def hernquist_density(r: np.ndarray) -> np.ndarray:
    return 1.0 / (2.0 * math.pi * r * (1.0 + r) ** 3)


def _nfw_tables(c: float):
    """Truncated NFW (r_s = 1, total mass M(<c) = 1, G = 1): radius grid,
    density, relative potential and the Eddington DF on an energy grid."""
    mu_c = math.log1p(c) - c / (1.0 + c)
    rho_s = 1.0 / (4.0 * math.pi * mu_c)
    r = np.logspace(-6, math.log10(c), 4000)
    rho = rho_s / (r * (1.0 + r) ** 2)
    m = (np.log1p(r) - r / (1.0 + r)) / mu_c
    # relative potential of the truncated sphere: psi(r) = 1/c + int_r^c m/r'^2
    integrand = m / (r * r)
    seg = 0.5 * (integrand[1:] + integrand[:-1]) * np.diff(r)
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    psi = 1.0 / c + tail
    # Eddington: f(E) = 1/(sqrt(8) pi^2) d/dE int_0^E drho/dpsi dpsi / sqrt(E - psi)
    lp, lr = psi[::-1], rho[::-1]                    # increasing psi
    drho = np.gradient(lr, lp)
    E = np.linspace(lp[0] * 1.0001, lp[-1] * 0.9999, 1500)
    I = np.empty_like(E)
    for k, e in enumerate(E):
        # substitution psi = E - t^2 removes the inverse square root
        t = np.linspace(0.0, math.sqrt(e - lp[0]), 400)
        ps = e - t * t
        I[k] = np.trapezoid(2.0 * np.interp(ps, lp, drho), t)
    f = np.gradient(I, E) / (math.sqrt(8.0) * math.pi ** 2)
    f = np.maximum(f, 0.0)
    return r, rho, psi, E, f


def nfw_halo(n: int, seed: int = 2, c: float = 10.0, ids: str = "arange") -> Particles:
    """Isolated NFW sphere (r_s = 1, G = 1, M(<c r_s) = 1) truncated at c r_s,
    velocities from a numerical Eddington inversion of the truncated profile."""
    rng = np.random.default_rng(seed)
    rg, rho, psi_g, E, f = _nfw_tables(c)
    mu_c = math.log1p(c) - c / (1.0 + c)
    m_g = (np.log1p(rg) - rg / (1.0 + rg)) / mu_c
    X = rng.random(n)
    r = np.interp(X, m_g, rg)
    pos = _isotropic(rng, r)
    psi = np.interp(r, rg, psi_g)
    emin, emax = E[0], E[-1]

    def df(e):
        return np.interp(np.clip(e, emin, emax), E, f) * (e > 0)

    v = _sample_speeds(rng, psi, df, float(psi_g.max()))
    vel = _isotropic(rng, v)
    mass = np.full(n, 1.0 / n)
    vc_rs = math.sqrt((math.log(2.0) - 0.5) / mu_c)    # circular speed at r_s
    return Particles(pos, vel, mass, _ids(rng, n, ids), 0.0,
                     {"kind": "nfw", "c": c, "rho_s": 1.0 / (4.0 * math.pi * mu_c),
                      "v_c_rs": vc_rs})


def nfw_density(r: np.ndarray, c: float = 10.0) -> np.ndarray:
    mu_c = math.log1p(c) - c / (1.0 + c)
    return 1.0 / (4.0 * math.pi * mu_c) / (r * (1.0 + r) ** 2)


# ------------------------------------------------------- timestep bins ---

def timestep_bins(p: Particles, density, sigma_over_m: float, n_ngb: int,
                  c_sidm: float = 0.1, target_active: float = 0.10,
                  n_bins: int = 8) -> tuple[np.ndarray, float]:
    """Power-of-two timestep bins for a halo.

    Each particle's admissible step is estimated from the analytic local
    density rho(r) and its own speed as t_i = (3 n_ngb c / 16) / (rho (sigma/m)
    2|v|) (the order-of-magnitude collision-time estimate of Sec. 4.4; it only
    shapes the synthetic bin distribution).  Bin b has step dt_max * 2**-b;
    a particle takes the coarsest bin with step <= t_i, clipped to
    [0, n_bins - 1].  ``dt_max`` is picked from a log grid so that the mean
    active fraction over a full cycle, mean_i 2**(b_i - (n_bins - 1)), is
    closest to ``target_active``.  Returns (bins int8, dt_max)."""
    r = np.linalg.norm(p.pos, axis=1)
    r = np.maximum(r, 1e-12)
    v = np.maximum(np.linalg.norm(p.vel, axis=1), 1e-12)
    t = (3.0 * n_ngb * c_sidm / 16.0) / (density(r) * sigma_over_m * 2.0 * v)
    lt = np.log2(t)
    sub = lt if lt.shape[0] <= 20000 else np.random.default_rng(0).choice(lt, 20000, replace=False)
    best = None
    for ldt in np.linspace(lt.min(), lt.max() + n_bins, 1000):
        b = np.ceil(ldt - sub).clip(0, n_bins - 1)
        frac = float(np.mean(np.exp2(b - (n_bins - 1))))
        score = abs(frac - target_active)
        if best is None or score < best[0]:
            best = (score, float(ldt))
    ldt = best[1]
    bins = np.ceil(ldt - lt).clip(0, n_bins - 1)
    return bins.astype(np.int8), float(2.0 ** ldt)


def eq18_bins(dt_limit: np.ndarray, target_active: float = 0.10, cycle: int = 100,
              max_bins: int = 40) -> tuple[np.ndarray, float]:
    """Power-of-two bins from per-particle Eq. 18 limits (Sec. 4.4), the
    harness rule of an individual-timestep code: particle i takes the
    smallest bin b >= 0 with dt_max 2^-b < dt_limit_i (strict), so every
    particle steps below its own limit and no bin is clipped.  dt_max is
    bisected (in log2) so that the mean active fraction over the first
    `cycle` finest steps is closest to target_active.  Infinite limits (no
    neighbour moving relative to the particle) take bin 0.  Returns (bins
    int8, dt_max)."""
    lim = np.asarray(dt_limit, np.float64)
    fin = np.isfinite(lim) & (lim > 0)
    l2 = np.log2(np.where(fin, lim, 1.0))

    def bins_for(ldt):
        # smallest b with ldt - b < l2, i.e. b = floor(ldt - l2) + 1, at least 0
        b = np.floor(ldt - l2) + 1.0
        return np.where(fin, np.clip(b, 0, max_bins - 1), 0).astype(np.int64)

    def frac(ldt):
        b = bins_for(ldt)
        period = np.left_shift(np.int64(1), int(b.max()) - b)
        return float(np.mean(np.ceil(cycle / period)) / cycle)

    lo, hi = float(l2[fin].min()) - 1.0, float(l2[fin].max()) + max_bins - 2.0
    for _ in range(60):          # frac decreases as dt_max grows
        mid = 0.5 * (lo + hi)
        if frac(mid) > target_active:
            lo = mid
        else:
            hi = mid
    ldt = lo if abs(frac(lo) - target_active) <= abs(frac(hi) - target_active) else hi
    return bins_for(ldt).astype(np.int8), float(2.0 ** ldt)


def active_at_step(bins: np.ndarray, s: int) -> np.ndarray:
    """Particle i is active at finest step s iff s is a multiple of
    2**(b_max - b_i) (bin 0 is the coarsest)."""
    bmax = int(bins.max())
    period = np.left_shift(1, (bmax - bins.astype(np.int64)))
    return (s % period == 0).astype(np.uint8)


# -------------------------------------------------------- named workloads ---

def box_32cubed(seed: int = 0) -> dict:
    """Uniform periodic unit box, N = 32^3, m = 1/N, sigma_1D = 1,
    N_ngb = 32, constant sigma/m = 1, every particle active, one step, with
    dt such that the mean scatter probability per particle is ~0.1 (rate
    rho (sigma/m) 4 sigma_1D / sqrt(pi))."""
    p = uniform_box(32 ** 3, 1.0, 1.0, seed)
    dt = 0.1 * math.sqrt(math.pi) / 4.0
    return {"name": "box-32^3", "particles": p, "n_ngb": 32, "sigma0": 1.0,
            "dt_max": dt, "bins": np.zeros(p.n, np.int8), "steps": 1,
            "seed": 0}


def hernquist_2pow20(seed: int = 1, n: int = 1 << 20) -> dict:
    """Isolated Hernquist halo, N = 2^20, N_ngb = 64, constant sigma/m = 1,
    power-of-two bins with ~10 % active per finest step, 100 steps."""
    p = hernquist_halo(n, seed)
    bins, dt_max = timestep_bins(p, hernquist_density, 1.0, 64)
    return {"name": f"hernquist-2^{int(math.log2(n))}", "particles": p, "n_ngb": 64,
            "sigma0": 1.0, "dt_max": dt_max, "bins": bins, "steps": 100, "seed": 0}


def _batch_member(args) -> dict:
    n, halo_seed, sigma0, n_ngb, key_seed = args
    p = hernquist_halo(n, halo_seed)
    bins, dt = timestep_bins(p, hernquist_density, sigma0, n_ngb)
    return {"particles": p, "bins": bins, "dt_max": dt, "sigma0": sigma0, "seed": key_seed}


def hernquist_batch(n_halos: int = 512, seed: int = 1000, log2_n=(12.0, 18.0),
                    sigma_range=(0.1, 10.0), n_ngb: int = 64, workers: int = 0) -> list:
    """Independent Hernquist haloes with N log-uniform in 2^[log2_n] and
    sigma/m log-uniform in sigma_range; halo k has seed seed + k, its own
    power-of-two bins and dt_max (10 % mean activity).  workers > 1 builds
    the haloes in that many spawned processes (same result: each halo
    depends only on its own seeds)."""
    rng = np.random.default_rng(seed)
    sizes = np.round(2.0 ** rng.uniform(log2_n[0], log2_n[1], n_halos)).astype(np.int64)
    sig = 10.0 ** rng.uniform(math.log10(sigma_range[0]), math.log10(sigma_range[1]), n_halos)
    jobs = [(int(sizes[k]), seed + 1 + k, float(sig[k]), n_ngb, seed + k) for k in range(n_halos)]
    if workers > 1 and n_halos > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batch_member, jobs, chunksize=8))
    return [_batch_member(j) for j in jobs]


def pack(haloes: list) -> tuple:
    """Concatenates haloes into one particle set; returns (Particles, offsets,
    bins) with halo k = particles [offsets[k], offsets[k+1])."""
    ps = [h["particles"] for h in haloes]
    off = np.zeros(len(ps) + 1, np.int64)
    off[1:] = np.cumsum([p.n for p in ps])
    cat = Particles(np.concatenate([p.pos for p in ps]), np.concatenate([p.vel for p in ps]),
                    np.concatenate([p.mass for p in ps]), np.concatenate([p.ids for p in ps]),
                    ps[0].box if ps else 0.0, {"kind": "batch"})
    bins = np.concatenate([h["bins"] for h in haloes]).astype(np.int8)
    return cat, off, bins
