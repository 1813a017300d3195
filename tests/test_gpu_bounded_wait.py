"""The resolver's wait is bounded.  When its pass limit runs out, the step
reports SIDM_ERR_DEVICE_LIMIT and the device stays usable.  Here the limit is
made to run out on purpose: one pass on a step whose kicks form long chains.
No fault is involved; the kernel stops after its passes and returns."""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def test_resolver_pass_limit_is_reported_and_the_device_stays_usable():
    p = I.hernquist_halo(20000, 61, ids="random")
    bins = np.zeros(p.n, np.int8)
    ctx = sidm.Context(n_ngb=32, max_resolver_passes=1)
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    with pytest.raises(sidm.SidmError) as e:
        ctx.step(4.0, None, bins, seed=62)          # P ~ 1 in the centre: chains of kicks
    assert e.value.status == sidm.ERR_DEVICE_LIMIT
    ctx.close()
    # a new context on the same device steps exactly as before
    ctx2 = sidm.Context(n_ngb=32)
    ctx2.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    st = ctx2.step(4.0, None, bins, seed=62)
    v, h = ctx2.velocities()
    ctx2.close()
    o = oracle.step(p.pos, p.vel, p.mass, p.ids, None, bins, 4.0, n_ngb=32, seed=62)
    assert st["n_accepted"] == o["n_pairs"] and st["max_multiplicity"] > 2
    assert np.array_equal(h, o["h"])
    assert np.array_equal(v, o["vel"])


def test_negative_pass_limit_is_rejected():
    with pytest.raises(sidm.SidmError) as e:
        sidm.Context(max_resolver_passes=-1)
    assert e.value.status == sidm.ERR_INVALID_ARG
