"""The no-allocation kick entry point (sidm_apply_pairs_noalloc).

Some callers cannot let a library allocate device memory: simulation codes
that reserve all GPU memory in their own pool at start-up, or that call in
from a place where a cudaMalloc would synchronise the device or is not
allowed.  For them the library applies accepted pairs with its scratch in
one fixed array inside the library.  These tests call that entry point
through the C ABI and check, on two calls in a row, that it gives the
velocities the regular step (sidm_step) gives for the same pairs, and bit
for bit the velocities of the oracle's sequential application of the same
records (ascending (ord, a, b), equal keys in the order given).  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu

# the tolerance of the step's parity tests: the kicks are bit-identical by
# construction; 1e-12 relative is the stated bound
REL_TOL = 1e-12


def _records(ab, ords, idx=None):
    """sidm_pair records; idx defaults to the ids (ids equal indices)."""
    rec = np.zeros(ab.shape[0], sidm.PAIR_DTYPE)
    rec["ord"] = ords
    rec["a"], rec["b"] = ab[:, 0], ab[:, 1]
    if idx is None:
        idx = ab
    rec["ia"], rec["ib"] = idx[:, 0].astype(np.int32), idx[:, 1].astype(np.int32)
    return rec


def _close(a, b):
    scale = np.maximum(np.abs(b), 1e-300)
    return float(np.max(np.abs(a - b) / scale)) <= REL_TOL


def _apply(rec, vel, mass, seed, step, stream="current"):
    import torch
    rec_d = torch.from_numpy(np.ascontiguousarray(rec).view(np.uint8)).cuda()
    vel_d = torch.from_numpy(np.ascontiguousarray(vel)).cuda()
    mass_d = torch.from_numpy(np.ascontiguousarray(mass)).cuda()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream().cuda_stream if stream == "current" else None
    st = sidm.sidm_apply_pairs_noalloc(rec_d, rec.shape[0], vel_d, mass_d, vel.shape[0], seed,
                                       step, s)
    assert st in (sidm.OK, sidm.WARN_DIRECTION)
    return vel_d.cpu().numpy()


def _oracle(orc, rec, vel, mass, seed, step):
    ab = np.stack([rec["a"], rec["b"]], 1)
    idx = np.stack([rec["ia"], rec["ib"]], 1)
    v, _ = orc.apply_pairs(vel, mass, rec["ord"], ab, idx, seed, step)
    return v


def test_noalloc_kicks_match_the_step_on_two_calls_in_a_row(orc):
    n = 30000
    p = I.uniform_box(n, 1.0, 1.0, 77)          # ids = 0..n-1 = indices
    bins = np.zeros(n, np.int8)
    seed = 4242
    ctx = sidm.Context(box=1.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    v_before = p.vel.copy()
    for call in range(2):
        step = ctx.step_counter
        ctx.step(0.3, None, bins, seed=seed)
        v_step, _ = ctx.velocities()
        ab, ords = ctx.pairs()
        assert ab.shape[0] > 500
        rec = _records(ab, ords)
        v_noalloc = _apply(rec, v_before, p.mass, seed, step)
        assert _close(v_noalloc, v_step), f"call {call}"
        assert np.array_equal(v_noalloc, _oracle(orc, rec, v_before, p.mass, seed, step)), call
        assert not np.array_equal(v_noalloc, v_before)
        v_before = v_step
    ctx.close()


def test_noalloc_serialises_repeated_records_like_the_oracle(orc):
    """A record given more than once is applied once per copy, one after the
    other (never twice in one round of the kick kernel)."""
    n = 20000
    p = I.uniform_box(n, 1.0, 1.0, 78, ids="random")
    rng = np.random.default_rng(5)
    o = orc.step(p.pos, p.vel, p.mass, p.ids, None, np.zeros(n, np.int8), 0.2, box=1.0, seed=9,
                 step=3)
    ab, ords = o["pairs_ab"], o["pairs_ord"]
    pos_of = {int(i): k for k, i in enumerate(p.ids)}
    idx = np.array([[pos_of[int(x)] for x in r] for r in ab], np.int64)
    rec = _records(ab, ords, idx)
    dup = rng.choice(rec.shape[0], 64, replace=False)
    rec = np.concatenate([rec, rec[dup], rec[dup[:8]]])
    rec = rec[rng.permutation(rec.shape[0])]
    v = _apply(rec, p.vel, p.mass, 9, 3)
    assert np.array_equal(v, _oracle(orc, rec, p.vel, p.mass, 9, 3))
    # without the copies it is the step's own result
    assert np.array_equal(_apply(_records(ab, ords, idx), p.vel, p.mass, 9, 3), o["vel"])


def test_noalloc_one_particle_in_many_pairs_on_the_default_stream(orc):
    """Particle 0 in 1500 pairs with random order keys (one kick per round),
    called on the legacy default stream (stream NULL)."""
    n = 4000
    rng = np.random.default_rng(6)
    vel = rng.normal(size=(n, 3))
    mass = rng.uniform(0.5, 2.0, n)
    m = 1500
    partner = rng.choice(np.arange(1, n), m, replace=False)
    ab = np.stack([np.zeros(m, np.uint32), partner.astype(np.uint32)], 1)
    ords = rng.integers(0, 1 << 63, m, dtype=np.int64).astype(np.uint64)
    rec = _records(ab, ords)
    v = _apply(rec, vel, mass, 11, 1 << 20, stream=None)
    assert np.array_equal(v, _oracle(orc, rec, vel, mass, 11, 1 << 20))
    # a second call in a row continues from the first call's velocities
    v2 = _apply(rec, v, mass, 11, (1 << 20) + 1, stream=None)
    assert np.array_equal(v2, _oracle(orc, rec, v, mass, 11, (1 << 20) + 1))


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_indices():
    import torch
    vel = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    mass = torch.ones(4, dtype=torch.float64, device="cuda")
    rec = np.zeros(1, sidm.PAIR_DTYPE)
    rec["a"], rec["b"], rec["ia"], rec["ib"] = 0, 1, 0, 1
    rec_d = torch.from_numpy(rec.view(np.uint8)).cuda()
    with pytest.raises(sidm.SidmError) as e:
        sidm.sidm_apply_pairs_noalloc(rec_d, 1, vel, mass, sidm.NOALLOC_MAX_PARTICLES + 1, 0, 0)
    assert e.value.status == sidm.ERR_TOO_LARGE
    with pytest.raises(sidm.SidmError) as e:
        sidm.sidm_apply_pairs_noalloc(rec_d, sidm.NOALLOC_MAX_PAIRS + 1, vel, mass, 4, 0, 0)
    assert e.value.status == sidm.ERR_TOO_LARGE
    bad = rec.copy()
    bad["ib"] = 7                                   # outside [0, n)
    with pytest.raises(sidm.SidmError) as e:
        sidm.sidm_apply_pairs_noalloc(torch.from_numpy(bad.view(np.uint8)).cuda(), 1, vel, mass,
                                      4, 0, 0)
    assert e.value.status == sidm.ERR_INVALID_ARG
    assert torch.count_nonzero(vel).item() == 0
