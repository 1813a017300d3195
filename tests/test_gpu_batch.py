"""Many haloes in one context (sidm_set_haloes / sidm_step_haloes).

Every halo of a batch must give, bit for bit, what a context holding that
halo alone gives with the same parameters: its own neighbour structure,
start radius, cross-section model, seed and step counter; no pair crosses
haloes.  One halo is also checked against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _params(h, k, step):
    return {"dt_max": h["dt_max"], "sigma0": h["sigma0"], "sigma_kind": k % 2, "w": 0.7,
            "seed": h["seed"], "step": step}


def _alone(h, k, starts, n_steps, n_ngb=64):
    p = h["particles"]
    ctx = sidm.Context(n_ngb=n_ngb, box=0.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    for t in range(n_steps):
        s = starts + t
        ctx.step_counter = s
        ctx.step(h["dt_max"], I.active_at_step(h["bins"], s), h["bins"], sigma0=h["sigma0"],
                 sigma_kind=k % 2, w=0.7, seed=h["seed"])
    v, hh = ctx.velocities()
    dl = ctx.timestep_limits()
    ctx.close()
    return v, hh, dl


def _batch(haloes, starts, n_steps, n_ngb=64, tune=None):
    p, off, bins = I.pack(haloes)
    ctx = sidm.Context(n_ngb=n_ngb, box=0.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.set_haloes(off)
    if tune:
        ctx.set_tuning(**tune)
    for t in range(n_steps):
        params = [_params(h, k, starts[k] + t) for k, h in enumerate(haloes)]
        act = np.concatenate([I.active_at_step(h["bins"], starts[k] + t) if h["particles"].n else
                              np.zeros(0, np.uint8) for k, h in enumerate(haloes)])
        ctx.step_haloes(params, act, bins)
    v, hh = ctx.velocities()
    dl = ctx.timestep_limits()
    ctx.close()
    return v, hh, dl, off


def _small_batch():
    haloes = I.hernquist_batch(10, seed=77, log2_n=(8.0, 13.0))
    # an empty halo and one with fewer particles than N_ngb + tol + 1
    tiny = I.hernquist_halo(20, 5)
    tb, td = I.timestep_bins(tiny, I.hernquist_density, 1.0, 64)
    empty = I.Particles(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0, np.uint32))
    haloes.insert(3, {"particles": empty, "bins": np.zeros(0, np.int8), "dt_max": 1.0,
                      "sigma0": 1.0, "seed": 5})
    haloes.append({"particles": tiny, "bins": tb, "dt_max": td, "sigma0": 2.0, "seed": 9})
    return haloes


def test_batch_equals_each_halo_alone():
    haloes = _small_batch()
    starts = [(3 * k) % 7 for k in range(len(haloes))]
    vb, hb, db, off = _batch(haloes, starts, 3)
    for k, h in enumerate(haloes):
        if h["particles"].n == 0:
            continue
        va, ha, da = _alone(h, k, starts[k], 3)
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(vb[sl], va), f"halo {k}: velocities"
        assert np.array_equal(hb[sl], ha), f"halo {k}: h"
        assert np.array_equal(db[sl], da), f"halo {k}: dt limits"


@pytest.mark.parametrize("run", [1, 16])
def test_search_runs_across_halo_boundaries(run):
    """A search warp takes runs of consecutive active queries, and a query
    whose predecessor in the run lies in the same halo first gathers within
    6/5 of that query's h.  Runs of 16 cross many halo boundaries of the
    batch (empty and tiny haloes among them); runs of 1 use no such radius.
    Both must give the default shape's results bit for bit."""
    haloes = _small_batch()
    starts = [(5 * k) % 7 for k in range(len(haloes))]
    ref = _batch(haloes, starts, 2)
    got = _batch(haloes, starts, 2, tune={"search_run": run})
    for a, b in zip(ref[:3], got[:3]):
        assert np.array_equal(a, b)


def test_batch_halo_matches_oracle():
    haloes = _small_batch()
    starts = [1] * len(haloes)
    vb, hb, db, off = _batch(haloes, starts, 2)
    k = 5
    h = haloes[k]
    p = h["particles"]
    vel, hh, dl = p.vel.copy(), np.zeros(p.n), np.full(p.n, np.inf)
    for t in range(2):
        s = 1 + t
        o = oracle.step(p.pos, vel, p.mass, p.ids, I.active_at_step(h["bins"], s), h["bins"],
                        h["dt_max"], n_ngb=64, sigma_kind=k % 2, sigma0=h["sigma0"], w=0.7,
                        seed=h["seed"], step=s, h_init=hh, dtlim_init=dl)
        vel, hh, dl = o["vel"], o["h"], o["dtlim"]
    sl = slice(off[k], off[k + 1])
    assert np.array_equal(vb[sl], vel)
    assert np.array_equal(hb[sl], hh)
    assert np.array_equal(db[sl], dl)


def test_set_haloes_validation():
    p = I.uniform_box(100, 1.0, 1.0, 3)
    ctx = sidm.Context(box=0.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    for bad in ([0, 50, 99], [1, 100], [0, 60, 40, 100], [0]):
        with pytest.raises(sidm.SidmError):
            ctx.set_haloes(bad)
    ctx.set_haloes([0, 40, 40, 100])
    with pytest.raises(sidm.SidmError):
        ctx.step_haloes([{"dt_max": 0.1}, {"dt_max": -1.0}, {"dt_max": 0.1}])
    ctx.close()


@pytest.fixture(scope="module")
def batch512():
    return I.hernquist_batch(512)


def test_hernquist_batch_512_sampled_haloes(batch512):
    """The many-halo workload (512 Hernquist haloes, N log-uniform in
    [2^12, 2^18], sigma/m log-uniform in [0.1, 10]) stepped as one batch;
    sampled haloes compared with the same haloes stepped alone."""
    haloes = batch512
    starts = [k % 4 for k in range(len(haloes))]
    vb, hb, db, off = _batch(haloes, starts, 1)
    for k in (0, 137, 301, 511):
        va, ha, da = _alone(haloes[k], k, starts[k], 1)
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(vb[sl], va), f"halo {k}"
        assert np.array_equal(hb[sl], ha), f"halo {k}"
        assert np.array_equal(db[sl], da), f"halo {k}"


def test_velocity_mirror_over_a_batch():
    """The velocity mirror (sidm_set_velocity_mirror) over many haloes in
    one context: after each multi-halo step it equals the full read-back,
    with an empty halo and a tiny one in the batch."""
    torch = pytest.importorskip("torch")
    haloes = _small_batch()
    p, off, bins = I.pack(haloes)
    ctx = sidm.Context(n_ngb=64, box=0.0, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.set_haloes(off)
    mirror = torch.from_numpy(p.vel.copy()).pin_memory().numpy()
    ctx.set_velocity_mirror(mirror)
    changed = 0
    for t in range(3):
        params = [_params(h, k, 1 + t) for k, h in enumerate(haloes)]
        act = np.concatenate([I.active_at_step(h["bins"], 1 + t) if h["particles"].n else
                              np.zeros(0, np.uint8) for k, h in enumerate(haloes)])
        ctx.step_haloes(params, act, bins)
        ctx.sync()
        v, _ = ctx.velocities()
        assert np.array_equal(mirror, v), t
        changed += ctx.changed()[0].size
    assert changed > 50
    ctx.close()
