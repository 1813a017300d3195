"""The no-allocation kick entry point (sidm_apply_pairs_noalloc).

Some callers cannot let a library allocate device memory: simulation codes
that reserve all GPU memory in their own pool at start-up, or that call in
from a place where a cudaMalloc would synchronise the device or is not
allowed.  For them the library applies accepted pairs with its scratch in
one fixed array inside the library.  These tests call that entry point
through the C ABI and check, on two calls in a row, that it gives the
velocities the regular step (sidm_step) gives for the same pairs.  The
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu

# the tolerance of the step's parity tests: the kicks are bit-identical by
# construction; 1e-12 relative is the stated bound
REL_TOL = 1e-12


def _records(ab, ords):
    """sidm_pair records for particles whose ids equal their indices."""
    rec = np.zeros(ab.shape[0], sidm.PAIR_DTYPE)
    rec["ord"] = ords
    rec["a"], rec["b"] = ab[:, 0], ab[:, 1]
    rec["ia"], rec["ib"] = ab[:, 0].astype(np.int32), ab[:, 1].astype(np.int32)
    return rec


def _close(a, b):
    scale = np.maximum(np.abs(b), 1e-300)
    return float(np.max(np.abs(a - b) / scale)) <= REL_TOL


def test_noalloc_kicks_match_the_step_on_two_calls_in_a_row():
    import torch
    n = 30000
    p = I.uniform_box(n, 1.0, 1.0, 77)          # ids = 0..n-1 = indices
    bins = np.zeros(n, np.int8)
    seed = 4242
    ctx = sidm.Context(box=1.0)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    mass_d = torch.from_numpy(p.mass).cuda()
    v_before = p.vel.copy()
    for call in range(2):
        step = ctx.step_counter
        ctx.step(0.3, None, bins, seed=seed)
        v_step, _ = ctx.velocities()
        ab, ords = ctx.pairs()
        assert ab.shape[0] > 500
        rec = torch.from_numpy(_records(ab, ords).view(np.uint8)).cuda()
        vel_d = torch.from_numpy(v_before).cuda()
        torch.cuda.synchronize()
        st = sidm.sidm_apply_pairs_noalloc(rec, ab.shape[0], vel_d, mass_d, n, seed, step,
                                           torch.cuda.current_stream().cuda_stream)
        assert st in (sidm.OK, sidm.WARN_DIRECTION)
        v_noalloc = vel_d.cpu().numpy()
        assert _close(v_noalloc, v_step), f"call {call}"
        assert not np.array_equal(v_noalloc, v_before)
        v_before = v_step
    ctx.close()


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
