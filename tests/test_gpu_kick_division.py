"""The kick's divisions by M = m_a + m_b (Eqs. 12-13) on extreme values.

The device divides by M from its correctly rounded reciprocal (Markstein's
correction, with a remainder check that keeps only the correctly rounded
quotient) where M and the dividend lie in [2^-500, 2^500), and with the
division elsewhere.  These tests apply kicks of disjoint pairs through the
no-allocation entry point, whose kick is the step's, on masses and
velocities that span both ranges, and compare every velocity bit for bit
with the oracle's kick (plain IEEE division).
"""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _records(n_pairs):
    rec = np.zeros(n_pairs, sidm.PAIR_DTYPE)
    a = 2 * np.arange(n_pairs, dtype=np.int64)
    rec["ord"] = np.arange(n_pairs)
    rec["a"], rec["b"] = a, a + 1
    rec["ia"], rec["ib"] = a.astype(np.int32), (a + 1).astype(np.int32)
    return rec


def _values(rng, n_pairs):
    """Masses and velocities over wide exponent ranges, both signs, with
    special cases: equal velocities (zero relative speed), zero components,
    masses far apart, powers of two."""
    n = 2 * n_pairs
    kind = rng.integers(0, 4, n_pairs)
    e_m = np.where(kind[:, None] == 0, rng.uniform(-30, 10, (n_pairs, 2)),
                   rng.uniform(-600, 600, (n_pairs, 2)))
    mass = (np.exp2(np.floor(e_m)) * rng.uniform(1.0, 2.0, (n_pairs, 2))).reshape(n)
    pow2 = rng.random(n) < 0.05
    mass[pow2] = np.exp2(np.floor(np.log2(mass[pow2])))
    e_v = np.where(kind[:, None, None] == 1, rng.uniform(-520, 400, (n_pairs, 2, 3)),
                   rng.uniform(-20, 20, (n_pairs, 2, 3)))
    vel = (np.exp2(e_v) * rng.choice([-1.0, 1.0], (n_pairs, 2, 3))).reshape(n, 3)
    same = np.flatnonzero(kind == 3)[::3]
    vel[2 * same + 1] = vel[2 * same]                 # zero relative speed
    vel[rng.random((n, 3)) < 0.02] = 0.0
    return mass, vel


@pytest.mark.parametrize("seed", [11, 12])
def test_kicks_on_extreme_values_are_bit_identical_to_the_oracle(seed):
    import torch
    rng = np.random.default_rng(seed)
    n_pairs = 20000
    mass, vel = _values(rng, n_pairs)
    rec = _records(n_pairs)
    vel_d = torch.from_numpy(vel.copy()).cuda()
    mass_d = torch.from_numpy(mass).cuda()
    rec_d = torch.from_numpy(rec.view(np.uint8)).cuda()
    philox_seed, step = 977 + seed, 5
    st = sidm.sidm_apply_pairs_noalloc(rec_d, n_pairs, vel_d, mass_d, 2 * n_pairs, philox_seed,
                                       step, torch.cuda.current_stream().cuda_stream)
    assert st in (sidm.OK, sidm.WARN_DIRECTION)
    got = vel_d.cpu().numpy()
    want = vel.copy()
    for k in range(n_pairs):
        a, b = 2 * k, 2 * k + 1
        e, _ = oracle.direction(philox_seed, step, a, b)
        want[a], want[b] = oracle.kick(mass[a], mass[b], vel[a], vel[b], e)
    assert np.all(np.isfinite(want))
    diff = np.flatnonzero(np.any(got.view(np.uint64) != want.view(np.uint64), axis=1))
    assert diff.size == 0, f"{diff.size} particles differ, first {diff[:5]}"
