"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The FP64 plain form must reproduce the oracle exactly: the same h for every
active particle, the same Eq. 18 limits, the same accepted pairs (ids and
order keys) and the same velocities.  The bound stated for velocities is
1e-12 relative; the path is built to be bit-identical, and these tests
assert bit equality (a relative-difference report is printed on failure).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _gpu_step(ctx, p, act, bins, dt_max, **kw):
    st = ctx.step(dt_max, act, bins, sigma0=kw.get("sigma0", 1.0),
                  sigma_kind=kw.get("sigma_kind", 0), w=kw.get("w", 1.0), seed=kw.get("seed", 0),
                  inelastic=kw.get("inelastic", 0.0))
    v, h = ctx.velocities()
    return {"vel": v, "h": h, "dtlim": ctx.timestep_limits(), "pairs": ctx.pairs(), "stats": st}


def _compare(g, o, act, what=""):
    act = np.ones(g["h"].shape[0], bool) if act is None else act.astype(bool)
    gs, os_ = g["stats"], o["stats"]
    assert gs["n_active"] == os_["n_active"], what
    assert gs["n_h_nonconv"] == os_["n_h_nonconv"], what
    bad = np.nonzero(g["h"][act] != o["h"][act])[0]
    assert bad.size == 0, f"{what}: h differs at {bad.size} particles, e.g. {g['h'][act][bad[:3]]} vs {o['h'][act][bad[:3]]}"
    assert gs["n_candidate_pairs"] == os_["n_candidate_pairs"], what
    assert gs["n_p_ge_1"] == os_["n_p_ge_1"], what
    ab, ords = g["pairs"]
    assert gs["n_accepted"] == o["n_pairs"], what
    assert np.array_equal(ab, o["pairs_ab"]), what
    assert np.array_equal(ords, o["pairs_ord"]), what
    dl_g, dl_o = g["dtlim"][act], o["dtlim"][act]
    assert np.array_equal(dl_g, dl_o), what
    if not np.array_equal(g["vel"], o["vel"]):
        rel = np.abs(g["vel"] - o["vel"]) / np.maximum(np.abs(o["vel"]), 1e-300)
        pytest.fail(f"{what}: velocities differ, max rel {rel.max():.3e}")
    # sum_p is a statistic: pairs whose draw is decided on the FP32 upper
    # bound contribute their FP32 estimate (relative error < 1e-5)
    assert math.isclose(gs["sum_p"], os_["sum_p"], rel_tol=1e-5, abs_tol=1e-30)
    assert abs(gs["e_after"] - os_["e_after"]) <= 1e-13 * abs(os_["e_after"]) + 1e-300


def run_pair(p, act, bins, dt_max, *, n_ngb=32, ngb_tol=5, kernel=0, fixed_h=0.0, steps=1,
             seed=0, sigma_kind=0, sigma0=1.0, w=1.0, c_sidm=0.1, device_inputs=False,
             pair_capacity=0, inelastic=0.0, overlap_table=None):
    ctx = sidm.Context(n_ngb=n_ngb, ngb_tol=ngb_tol, c_sidm=c_sidm, box=p.box, kernel=kernel,
                       fixed_h=fixed_h, pair_capacity=pair_capacity,
                       estimator=int(overlap_table is not None))
    if overlap_table is not None:
        ctx.set_overlap_table(overlap_table)
    if device_inputs:
        import torch
        ctx.set_particles(torch.from_numpy(p.pos).cuda(), torch.from_numpy(p.vel).cuda(),
                          torch.from_numpy(p.ids.astype(np.int32)).cuda(),
                          mass=torch.from_numpy(p.mass).cuda())
    else:
        ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    vel = p.vel.copy()
    h = np.zeros(p.n)
    dl = np.full(p.n, np.inf)
    for k in range(steps):
        a = act(k) if callable(act) else act
        o = oracle.step(p.pos, vel, p.mass, p.ids, a, bins, dt_max, n_ngb=n_ngb, ngb_tol=ngb_tol,
                        c_sidm=c_sidm, box=p.box, kernel=kernel, fixed_h=fixed_h,
                        sigma_kind=sigma_kind, sigma0=sigma0, w=w, inelastic=inelastic,
                        overlap_table=overlap_table, seed=seed, step=k, h_init=h, dtlim_init=dl)
        g = _gpu_step(ctx, p, a, bins, dt_max, sigma_kind=sigma_kind, sigma0=sigma0, w=w, seed=seed,
                      inelastic=inelastic)
        _compare(g, o, a, f"step {k}")
        vel, h, dl = o["vel"], o["h"], o["dtlim"]
        # outputs of inactive particles keep their previous values
        assert np.array_equal(g["h"], h) and np.array_equal(g["dtlim"], dl)
    ctx.close()
    return g, o


def test_box_small_all_active():
    p = I.uniform_box(4096, 1.0, 1.0, 3)
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 0.05)
    assert o["n_pairs"] > 50


@pytest.mark.parametrize("inelastic", [0.5, 1.0])
def test_inelastic_scatters_match_the_oracle(inelastic):
    """eps = 1 - inelastic < 1 (Sec. 4.1): same pairs, bit-identical velocities
    over several steps (eps = 0: the pair leaves at its centre-of-momentum
    velocity)."""
    p = I.uniform_box(5000, 1.0, 1.0, 17, ids="random")
    bins = np.zeros(p.n, np.int8)
    g, o = run_pair(p, None, bins, 0.15, steps=3, seed=4, inelastic=inelastic)
    assert o["n_pairs"] > 100
    assert g["stats"]["e_after"] < g["stats"]["e_before"]


def test_box_32cubed_workload():
    w = I.box_32cubed()
    p = w["particles"]
    g, o = run_pair(p, None, w["bins"], w["dt_max"])
    assert 1400 < o["n_pairs"] < 1900
    assert abs(g["stats"]["e_after"] - g["stats"]["e_before"]) <= 1e-13 * g["stats"]["e_before"]


def test_halo_partial_activity_random_ids_unequal_masses():
    p = I.hernquist_halo(20000, 5, ids="random")
    rng = np.random.default_rng(1)
    p.mass = p.mass * rng.uniform(0.5, 1.5, p.n)
    bins = rng.integers(0, 4, p.n).astype(np.int8)
    act = (rng.random(p.n) < 0.3).astype(np.uint8)
    run_pair(p, act, bins, 0.2, n_ngb=64)


def test_large_neighbour_number_with_the_smallest_window():
    # K = N_ngb + tol + 1 = 206 exceeds the 127 other particles of a
    # 128-particle window, which then cannot bound the search radius: the
    # launch takes the 256-particle window instead, with the same results
    p = I.hernquist_halo(20000, 7, ids="random")
    rng = np.random.default_rng(2)
    act = (rng.random(p.n) < 0.2).astype(np.uint8)
    bins = np.zeros(p.n, np.int8)
    ctx = sidm.Context(n_ngb=200, ngb_tol=5)
    ctx.set_tuning(search_window=128)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    o = oracle.step(p.pos, p.vel, p.mass, p.ids, act, bins, 2.0, n_ngb=200, ngb_tol=5, seed=0,
                    step=0)
    g = _gpu_step(ctx, p, act, bins, 2.0)
    assert ctx.tuning["search_window"] == 128
    ctx.close()
    _compare(g, o, act)
    assert o["n_pairs"] > 100


def test_coincident_positions_match_the_oracle():
    # groups of 8 particles at identical positions (zero separations in the
    # window radius, the gather and the bisection) and one clump of 121, more
    # than N_ngb + tol, whose members can reach no admissible count
    p = I.uniform_box(4096, 1.0, 1.0, 41, ids="random")
    p.pos[:] = np.repeat(p.pos[::8].copy(), 8, axis=0)[:p.n]
    p.pos[-120:] = p.pos[-121]
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 0.02, seed=5)
    assert o["stats"]["n_h_nonconv"] > 120 and o["n_pairs"] > 1000


def test_halo_far_from_the_origin_matches_the_oracle():
    # at |x| ~ 3e5 the FP32 copies resolve ~0.02, a good part of the
    # spacing: many certified bounds are ambiguous and the exact FP64 tests
    # decide
    q = I.hernquist_halo(20000, 9, ids="random")
    q.pos = q.pos + np.array([1.0e5, -2.0e5, 3.0e5])
    act = (np.random.default_rng(3).random(q.n) < 0.3).astype(np.uint8)
    g, o = run_pair(q, act, np.zeros(q.n, np.int8), 5.0, seed=6)
    assert o["n_pairs"] > 300


def test_yukawa_tophat_box():
    p = I.uniform_box(3000, 2.0, 1.5, 4, ids="random")
    run_pair(p, None, np.zeros(p.n, np.int8), 0.3, kernel=1, sigma_kind=1, sigma0=5.0, w=1.2)


def test_fixed_h_hook():
    p = I.uniform_box(2000, 1.0, 1.0, 5)
    run_pair(p, None, np.zeros(p.n, np.int8), 0.02, fixed_h=0.12)


@pytest.mark.parametrize("n", [1, 2, 5, 38, 39, 40, 70, 1000, 1025, 4097])
@pytest.mark.parametrize("box", [1.0, 0.0])
def test_ragged_and_tiny_sizes(n, box):
    p = I.uniform_box(n, 1.0, 1.0, 100 + n)
    p.box = box
    run_pair(p, None, np.zeros(n, np.int8), 0.1)


def test_every_kick_warp_busy_with_pending_pairs():
    """More pending pairs than the kick application's cooperative grid has
    warps to spare (at most 7 x 32 x 1184 = 265,216 on a B300): every warp
    holds pending pairs, so each thread applies its share of the isolated
    pairs after its pending ones.  An all-active periodic box of 2^20
    particles at unit density, with dt for about 1.2 expected scatters per
    particle (~6e5 accepted pairs, most sharing a particle with another),
    against the oracle."""
    n = 1 << 20
    p = I.uniform_box(n, 1.0, 1.0, 31)
    g, o = run_pair(p, None, np.zeros(n, np.int8), 1.2 * math.sqrt(math.pi) / 4.0)
    assert o["n_pairs"] > 400_000


def test_no_active_particles():
    p = I.uniform_box(3000, 1.0, 1.0, 6)
    g, o = run_pair(p, np.zeros(p.n, np.uint8), np.zeros(p.n, np.int8), 0.1)
    assert o["n_pairs"] == 0 and np.array_equal(g["vel"], p.vel)


def test_several_steps_with_changing_activity():
    p = I.uniform_box(6000, 1.0, 1.0, 7, ids="random")
    rng = np.random.default_rng(2)
    masks = [(rng.random(p.n) < f).astype(np.uint8) for f in (1.0, 0.3, 0.05, 0.6)]
    bins = rng.integers(0, 3, p.n).astype(np.int8)
    run_pair(p, lambda k: masks[k], bins, 0.15, steps=4, seed=12345678901)


def test_lattice_without_admissible_count():
    g_ = np.arange(8) / 8.0
    x, y, z = np.meshgrid(g_, g_, g_, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    n = pos.shape[0]
    p = I.Particles(pos, np.random.default_rng(0).normal(size=(n, 3)), np.full(n, 1.0 / n),
                    np.arange(n, dtype=np.uint32), 1.0)
    g, o = run_pair(p, None, np.zeros(n, np.int8), 0.1, n_ngb=22, ngb_tol=1)
    assert o["stats"]["n_h_nonconv"] == n
    assert g["stats"]["return"] & sidm.WARN_H_NOT_CONVERGED


def test_probabilities_above_one():
    p = I.uniform_box(2000, 1.0, 1.0, 8)
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 20.0, pair_capacity=200000)
    assert o["stats"]["n_p_ge_1"] > 0
    assert g["stats"]["return"] & sidm.WARN_P_GE_1


def test_full_pair_buffer_is_reported_and_nothing_is_kicked():
    """A bounded buffer that fills makes the step return SIDM_ERR_DEVICE_LIMIT
    and leaves the velocities untouched (no partial application)."""
    p = I.uniform_box(3000, 1.0, 1.0, 12)
    ctx = sidm.Context(box=1.0, pair_capacity=5)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    with pytest.raises(sidm.SidmError) as e:
        ctx.step(0.5)
    assert e.value.status == sidm.ERR_DEVICE_LIMIT
    v, _ = ctx.velocities()
    assert np.array_equal(v, p.vel)
    ctx.close()


def test_pairs_at_zero_relative_speed_match_the_oracle():
    """Half the particles at rest and 500 pairs of bit-equal moving velocities:
    g(0) = 0 makes P_pair exactly zero for those pairs.  They are rejected
    without the exact FP64 pass; deferring them all would overflow this pair
    buffer, which holds about ten steps' worth of accepted pairs."""
    p = I.uniform_box(6000, 1.0, 1.0, 14, ids="random")
    h = p.n // 2
    p.vel[:h] = 0.0
    p.vel[h:h + 500] = p.vel[h + 500:h + 1000]
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 0.1, steps=3, seed=2, pair_capacity=p.n)
    assert o["n_pairs"] > 50


@pytest.mark.parametrize("sigma_kind", [0, 1])
def test_zero_cross_section_scatters_nothing(sigma_kind):
    """sigma0 = 0: every P_pair is exactly zero, nothing is deferred (a
    five-entry buffer suffices) and the Eq. 18 limits are infinite."""
    p = I.uniform_box(3000, 1.0, 1.0, 15)
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 0.5, sigma_kind=sigma_kind, sigma0=0.0,
                    pair_capacity=5)
    assert o["n_pairs"] == 0 and g["stats"]["n_accepted"] == 0
    assert np.array_equal(g["vel"], p.vel)
    assert np.all(np.isinf(g["dtlim"]))


def test_device_inputs_match_host_inputs():
    import torch
    p = I.uniform_box(5000, 1.0, 1.0, 9)
    run_pair(p, None, np.zeros(p.n, np.int8), 0.1, device_inputs=True)


def test_resume_is_bit_identical():
    p = I.uniform_box(4000, 1.0, 1.0, 10, ids="random")
    bins = np.zeros(p.n, np.int8)
    a = sidm.Context(box=1.0)
    a.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    a.step(0.2, None, bins, seed=9)
    v1, _ = a.velocities()
    a.step(0.2, None, bins, seed=9)
    v2, _ = a.velocities()
    b = sidm.Context(box=1.0)
    b.set_particles(p.pos, v1, p.ids, mass=p.mass)
    b.step_counter = 1
    b.step(0.2, None, bins, seed=9)
    v2b, _ = b.velocities()
    assert np.array_equal(v2, v2b) and not np.array_equal(v1, v2)


def test_invalid_inputs_are_rejected():
    ctx = sidm.Context(box=1.0)
    with pytest.raises(sidm.SidmError) as e:
        ctx.step(0.1)
    assert e.value.status == sidm.ERR_NOT_READY
    p = I.uniform_box(100, 1.0, 1.0, 11)
    bad = p.pos.copy()
    bad[3, 1] = 1.0
    with pytest.raises(sidm.SidmError) as e:
        ctx.set_particles(bad, p.vel, p.ids, mass=p.mass)
    assert e.value.status == sidm.ERR_INVALID_ARG
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    for dt in (0.0, -1.0, float("inf")):
        with pytest.raises(sidm.SidmError):
            ctx.step(dt)
    with pytest.raises(sidm.SidmError):
        ctx.step(0.1, sigma_kind=1, w=0.0)


@pytest.fixture(scope="module")
def hernquist_full():
    return I.hernquist_2pow20()


@pytest.mark.parametrize("s", [0, 1, 4])
def test_hernquist_2pow20_full_size(hernquist_full, s):
    """The halo workload at full size (N = 2^20, N_ngb = 64, open boundaries,
    power-of-two bins) in the configuration the benchmark times: a captured
    step graph with autotuned launch shapes.  Step 0 of the bin cycle has
    every particle active (~2e5 accepted pairs, the longest kick chains)."""
    w = hernquist_full
    p, bins = w["particles"], w["bins"]
    act = I.active_at_step(bins, s)
    ctx = sidm.Context(n_ngb=64, box=0.0, use_graph=True)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.step_counter = s
    ctx.autotune([sidm.HaloParams(w["dt_max"], sidm.SigmaModel(0, 1.0, 1.0), w["seed"], s)],
                 I.active_at_step(bins, 1), bins, reps=1)
    o = oracle.step(p.pos, p.vel, p.mass, p.ids, act, bins, w["dt_max"], n_ngb=64, seed=w["seed"],
                    step=s)
    g = _gpu_step(ctx, p, act, bins, w["dt_max"], seed=w["seed"])
    assert ctx.graph_state == 1
    _compare(g, o, act, f"hernquist step {s}")
    ctx.close()


def test_eq18_bins_from_the_oracle_limits_keep_every_pair_below_one():
    """A halo whose bins come from its own Eq. 18 limits (Sec. 4.4; the
    oracle's limits of an all-active step, smallest bin below each limit):
    several steps of the hierarchy match the oracle bit for bit, and no pair
    reaches P = 1."""
    p = I.hernquist_halo(1 << 14, 31, ids="random")
    o0 = oracle.step(p.pos, p.vel, p.mass, p.ids, None, np.zeros(p.n, np.int8), 1e-3, n_ngb=32,
                     seed=1)
    bins, dt_max = I.eq18_bins(o0["dtlim"], cycle=16)
    assert int(bins.max()) >= 3
    stats = []
    ctx = sidm.Context(n_ngb=32)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    vel, h, dl = p.vel.copy(), np.zeros(p.n), np.full(p.n, np.inf)
    for k in range(6):
        a = I.active_at_step(bins, k)
        o = oracle.step(p.pos, vel, p.mass, p.ids, a, bins, dt_max, n_ngb=32, seed=5, step=k,
                        h_init=h, dtlim_init=dl)
        g = _gpu_step(ctx, p, a, bins, dt_max, seed=5)
        _compare(g, o, a, f"step {k}")
        stats.append(g["stats"])
        vel, h, dl = o["vel"], o["h"], o["dtlim"]
    ctx.close()
    assert sum(st["n_accepted"] for st in stats) > 100
    assert all(st["n_p_ge_1"] == 0 for st in stats)


def test_tabulated_cross_section_matches_the_oracle():
    """Tabulated sigma/m(v), linear in log v (Sec. 4.1), on a halo with
    partial activity: h, accepted pairs and velocities equal the oracle's;
    the Eq. 18 limits agree to the last bits (the device and the host take
    their own logarithm of v)."""
    p = I.hernquist_halo(20000, 8, ids="random")
    rng = np.random.default_rng(9)
    tv = np.sort(10 ** rng.uniform(-2.0, 1.0, 16))
    ts = 10 ** rng.uniform(-1.0, 1.0, 16)
    bins = rng.integers(0, 4, p.n).astype(np.int8)
    ctx = sidm.Context(n_ngb=32, box=0.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    ctx.set_sigma_table(tv, ts)
    vel, h, dl = p.vel.copy(), np.zeros(p.n), np.full(p.n, np.inf)
    total = 0
    for k in range(3):
        act = I.active_at_step(bins, k)
        o = oracle.step(p.pos, vel, p.mass, p.ids, act, bins, 2.0, n_ngb=32, sigma_kind=2,
                        table=(tv, ts), seed=12, step=k, h_init=h, dtlim_init=dl)
        st = ctx.step(2.0, act, bins, sigma_kind=sidm.SIGMA_TABLE, seed=12)
        gv, gh = ctx.velocities()
        ab, ords = ctx.pairs()
        assert np.array_equal(gh, o["h"])
        assert np.array_equal(ab, o["pairs_ab"][: o["n_pairs"]])
        assert np.array_equal(ords, o["pairs_ord"][: o["n_pairs"]])
        assert np.array_equal(gv, o["vel"])
        gl = ctx.timestep_limits()
        fin = np.isfinite(o["dtlim"])
        assert np.array_equal(np.isfinite(gl), fin)
        assert np.allclose(gl[fin], o["dtlim"][fin], rtol=1e-14, atol=0)
        assert st["n_accepted"] == o["n_pairs"]
        total += o["n_pairs"]
        vel, h, dl = o["vel"], o["h"], o["dtlim"]
    assert total > 200
    ctx.close()


def test_sigma_table_validation():
    ctx = sidm.Context()
    p = I.uniform_box(500, 1.0, 1.0, 1)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    with pytest.raises(sidm.SidmError):      # no table yet
        ctx.step(0.1, sigma_kind=sidm.SIGMA_TABLE)
    for v, s in (([1.0], [1.0]), ([1.0, 1.0], [1.0, 2.0]), ([2.0, 1.0], [1.0, 1.0]),
                 ([0.0, 1.0], [1.0, 1.0]), ([1.0, 2.0], [1.0, -1.0]),
                 ([1.0, 1.0 + 1e-9], [1.0, 1.0])):
        with pytest.raises(sidm.SidmError):
            ctx.set_sigma_table(np.array(v), np.array(s))
    ctx.set_sigma_table(np.array([0.5, 2.0]), np.array([1.0, 3.0]))
    ctx.step(0.1, sigma_kind=sidm.SIGMA_TABLE, stats=False)
    ctx.close()


@pytest.fixture(scope="module")
def ov_tables():
    return {k: oracle.overlap_table(32, 128, kernel=k) for k in (0, 1)}


def test_overlap_estimator_box_all_active(ov_tables):
    """Kernel-overlap estimator (Eq. 15, Appendix A) in a periodic box: h of
    every particle, pairs (r_ij < h_i + h_j) and velocities equal the
    oracle's over several steps."""
    p = I.uniform_box(5000, 1.0, 1.0, 41, ids="random")
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 0.05, steps=3, seed=6,
                    overlap_table=ov_tables[0])
    assert o["n_pairs"] > 100


def test_overlap_estimator_halo_partial_activity(ov_tables):
    """Inactive neighbours enter with their own h (found for every particle);
    unequal masses, random ids, power-of-two bins."""
    p = I.hernquist_halo(15000, 42, ids="random")
    rng = np.random.default_rng(43)
    p.mass[:] = p.mass * rng.uniform(0.5, 2.0, p.n)
    bins = rng.integers(0, 4, p.n).astype(np.int8)
    g, o = run_pair(p, lambda k: I.active_at_step(bins, k), bins, 2.0, n_ngb=32, steps=3,
                    seed=7, overlap_table=ov_tables[0])
    assert o["n_pairs"] > 30


def test_overlap_estimator_fixed_h_tophat(ov_tables):
    p = I.uniform_box(3000, 1.0, 1.0, 44)
    g, o = run_pair(p, None, np.zeros(p.n, np.int8), 0.05, fixed_h=0.08, kernel=1,
                    overlap_table=ov_tables[1])
    assert o["n_pairs"] > 50


def test_overlap_estimator_needs_its_table():
    p = I.uniform_box(500, 1.0, 1.0, 45)
    ctx = sidm.Context(box=1.0, estimator=sidm.ESTIMATOR_OVERLAP)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    with pytest.raises(sidm.SidmError) as e:
        ctx.step(0.1)
    assert e.value.status == sidm.ERR_NOT_READY
    ctx.set_overlap_table(sidm.sidm_overlap_table(0, 8, 32))
    ctx.step(0.1, stats=False)
    ctx.close()
