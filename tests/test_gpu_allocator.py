"""Device memory through the caller's allocator (sidm_config.alloc / free,
the module's buffers living in the host code's pool, Sec. 4.6): with
PyTorch's caching allocator every device buffer of the context comes from
torch, the results are bit-identical to a context on cudaMalloc, and all of
it goes back when the context is destroyed."""
import numpy as np
import pytest

from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

pytestmark = pytest.mark.gpu


def _run(ctx, p, bins, steps=3):
    out = []
    for s in range(steps):
        st = ctx.step(0.05, I.active_at_step(bins, s), bins, seed=17)
        v, h = ctx.velocities()
        out.append((v, h, ctx.pairs(), ctx.timestep_limits(), st["n_accepted"]))
    return out


def test_torch_allocator_holds_every_buffer_and_results_are_unchanged():
    import torch
    torch.cuda.init()
    p = I.hernquist_halo(1 << 17, 3)
    bins, _ = I.timestep_bins(p, I.hernquist_density, 1.0, 32)
    n = p.n
    # every kernel loaded once (module loading takes device memory too)
    ref = sidm.Context(n_max=n)
    ref.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    want = _run(ref, p, bins)
    ref.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    ctx = sidm.Context(n_max=n, allocator="torch")
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    got = _run(ctx, p, bins)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    held = torch.cuda.memory_allocated() - alloc0
    cap = sidm.sidm_context_bytes(ctx.cfg, n)
    assert held >= cap                           # the capacity buffers and the tree
    # device memory taken outside torch's pool while the context lives: none
    # beyond allocation granularity
    outside = (free0 - free1) - (torch.cuda.memory_reserved() - res0)
    assert outside < 16 << 20, outside
    assert sum(w[4] for w in want) > 0
    for (v, h, (ab, o), d, k), (v2, h2, (ab2, o2), d2, k2) in zip(want, got):
        assert k == k2
        assert np.array_equal(v, v2) and np.array_equal(h, h2) and np.array_equal(d, d2)
        assert np.array_equal(ab, ab2) and np.array_equal(o, o2)
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0


def test_autotune_and_tables_use_the_allocator_too():
    import torch
    p = I.uniform_box(4096, 1.0, 1.0, 4)
    ctx = sidm.Context(box=1.0, allocator="torch")
    ctx.set_particles(p.pos, p.vel, p.ids, mass=p.mass)
    a0 = torch.cuda.memory_allocated()
    ctx.set_sigma_table(np.array([0.1, 1.0, 10.0]), np.array([2.0, 1.0, 0.5]))
    a1 = torch.cuda.memory_allocated()
    assert a1 > a0
    prm = [sidm.HaloParams(0.05, sidm.SigmaModel(sidm.SIGMA_TABLE, 0.0, 1.0), 1, 0)]
    torch.cuda.reset_peak_memory_stats()
    ctx.autotune(prm, None, None, reps=1)
    # the saved state (5 doubles per particle) came from torch and went back
    assert torch.cuda.max_memory_allocated() >= a1 + 5 * 8 * p.n
    assert torch.cuda.memory_allocated() == a1
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() < a0


def test_allocator_that_fails_gives_oom_not_a_crash():
    calls = []

    @sidm.ALLOC_FN
    def refuse(nbytes, stream, user):
        calls.append(nbytes)
        return None

    @sidm.FREE_FN
    def never(ptr, stream, user):
        raise AssertionError("nothing was allocated")

    cfg = sidm.sidm_default_config()
    cfg.n_max = 1000
    cfg.alloc, cfg.free = refuse, never
    with pytest.raises(sidm.SidmError) as e:
        sidm.sidm_create(cfg)
    assert e.value.status == sidm.ERR_OOM and calls
