"""The NFW halo at the benchmark's full size (N = 2^23, c = 10, Yukawa-like
sigma0/m = 1 with w = v_c(r_s), N_ngb = 64, open boundaries, power-of-two
bins) in the launch configuration the benchmark times: a captured step
graph with autotuned launch shapes.  The oracle covers a sampled active
set so that its step over the whole halo stays short: 448 particles spread
from the centre to the outskirts (every (N/448)-th by distance from the
centre) and the 64 innermost ones, which are each other's neighbours.
Every neighbour radius, accepted pair, velocity and Eq. 18 limit of the
step must equal the oracle's (FP64 plain form), and the FP32-split form
must accept the same pairs (Sec. 4.2-4.5, Eqs. 15-18)."""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

from test_gpu_parity import _compare, _gpu_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nfw_full():
    p = I.nfw_halo(1 << 23, 2)
    bins, dt = I.timestep_bins(p, I.nfw_density, 1.0, 64)
    r = np.linalg.norm(p.pos - p.pos.mean(0), axis=1)
    order = np.argsort(r)
    act = np.zeros(p.n, np.uint8)
    act[order[:: p.n // 448][:448]] = 1
    act[order[:64]] = 1
    return p, bins, dt, act


def _context(p, bins, dt, w, precision):
    ctx = sidm.Context(n_ngb=64, box=0.0, use_graph=True, precision=precision)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.step_counter = 1
    ctx.autotune([sidm.HaloParams(dt, sidm.SigmaModel(sidm.SIGMA_YUKAWA, 1.0, w), 7, 1)],
                 I.active_at_step(bins, 1), bins, reps=1)
    return ctx


def test_nfw_2pow23_sampled_active_set(nfw_full):
    p, bins, dt, act = nfw_full
    w = p.meta["v_c_rs"]
    o = oracle.step(p.pos, p.vel, p.mass, p.ids, act, bins, dt, n_ngb=64, sigma_kind=1,
                    sigma0=1.0, w=w, seed=7, step=1)
    assert o["n_pairs"] > 100
    ctx = _context(p, bins, dt, w, sidm.FP64_PLAIN)
    g = _gpu_step(ctx, p, act, bins, dt, sigma_kind=1, sigma0=1.0, w=w, seed=7)
    assert ctx.graph_state == 1
    _compare(g, o, act, "nfw 2^23, FP64 plain")
    ctx.close()
    split = _context(p, bins, dt, w, sidm.FP32_SPLIT)
    gs = _gpu_step(split, p, act, bins, dt, sigma_kind=1, sigma0=1.0, w=w, seed=7)
    ab, ords = gs["pairs"]
    assert np.array_equal(ab, o["pairs_ab"]) and np.array_equal(ords, o["pairs_ord"])
    split.close()
