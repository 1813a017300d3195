"""The four-function interface of a scattering model (Sec. 4.6: scatter,
get_state, set_state, overwrite_state) as a device-side template
(include/sidm_model.cuh).  tests/model_ext.cu writes two models against it,
as a host code would, and is compiled here with nvcc:
  * UserElastic, its own restatement of the elastic isotropic scatter
    (Sec. 4.1): applied to the accepted pairs of an oracle step, it gives the
    oracle's velocities bit for bit;
  * CountingElastic, the same with per-particle state the library does not
    know (a scatter count): the counts equal each particle's number of
    accepted pairs, and the velocities are again the oracle's.
The built-in model (IsotropicKick, which the scattering step itself uses)
through the same template also matches the oracle, elastic and inelastic."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_2607_05504_b300 import build as B
from paper_2607_05504_b300 import inputs as I
from paper_2607_05504_b300 import sidm

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _compile(out_dir) -> str:
    so = os.path.join(str(out_dir), "libmodel_ext.so")
    subprocess.check_call([B.NVCC, *B.ARCH, "-O3", "-std=c++17", "-fmad=false", "-shared",
                           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                           os.path.join(HERE, "model_ext.cu"), "-o", so])
    return so


def test_model_extension_builds_for_sm_103a(tmp_path):
    so = _compile(tmp_path)
    L = C.CDLL(so)
    for name in ("ext_apply_elastic", "ext_apply_counting", "ext_apply_builtin",
                 "ext_scratch_bytes"):
        assert hasattr(L, name)
    L.ext_scratch_bytes.restype = C.c_size_t
    L.ext_scratch_bytes.argtypes = [C.c_int64, C.c_int64]
    assert L.ext_scratch_bytes(1000, 100) >= 4 * 1000 * 4 + 100 * 40


@pytest.fixture(scope="module")
def ext(tmp_path_factory):
    L = C.CDLL(_compile(tmp_path_factory.mktemp("model")))
    vp, i64, u64 = C.c_void_p, C.c_int64, C.c_uint64
    L.ext_scratch_bytes.restype = C.c_size_t
    L.ext_scratch_bytes.argtypes = [i64, i64]
    L.ext_apply_elastic.argtypes = [vp, i64, vp, vp, i64, u64, u64, vp, C.c_size_t, vp]
    L.ext_apply_counting.argtypes = [vp, i64, vp, vp, vp, i64, u64, u64, vp, C.c_size_t, vp]
    L.ext_apply_builtin.argtypes = [vp, i64, vp, vp, i64, u64, u64, C.c_double, vp, C.c_size_t,
                                    vp]
    return L


def _step_pairs(orc, p, seed, step, dt=0.6, inelastic=0.0):
    o = orc.step(p.pos, p.vel, p.mass, p.ids, None, np.zeros(p.n, np.int8), dt, box=p.box,
                 seed=seed, step=step, inelastic=inelastic)
    pos_of = {int(i): k for k, i in enumerate(p.ids)}
    idx = np.array([[pos_of[int(x)] for x in r] for r in o["pairs_ab"]], np.int32)
    rec = np.zeros(idx.shape[0], sidm.PAIR_DTYPE)
    rec["ord"] = o["pairs_ord"]
    rec["a"], rec["b"] = o["pairs_ab"][:, 0], o["pairs_ab"][:, 1]
    rec["ia"], rec["ib"] = idx[:, 0], idx[:, 1]
    return o, rec


@pytest.mark.gpu
def test_user_models_through_the_interface_match_the_oracle(orc, ext):
    import torch
    p = I.uniform_box(20000, 1.0, 1.0, 91, ids="random")
    p.mass = np.random.default_rng(92).uniform(0.5, 2.0, p.n) / p.n
    stream = torch.cuda.current_stream().cuda_stream
    vel = p.vel.copy()
    for call, (seed, step) in enumerate(((5, 0), (5, 1))):
        q = I.Particles(p.pos, vel, p.mass, p.ids, p.box, p.meta)
        o, rec = _step_pairs(orc, q, seed, step)
        mult = np.bincount(np.concatenate([rec["ia"], rec["ib"]]), minlength=p.n)
        assert rec.shape[0] > 1000 and mult.max() >= 3        # pairs that share particles
        nb = ext.ext_scratch_bytes(p.n, rec.shape[0])
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        rec_d = torch.from_numpy(rec.view(np.uint8)).cuda()
        mass_d = torch.from_numpy(p.mass).cuda()
        v1 = torch.from_numpy(vel).cuda()
        assert ext.ext_apply_elastic(rec_d.data_ptr(), rec.shape[0], v1.data_ptr(),
                                     mass_d.data_ptr(), p.n, seed, step, scratch.data_ptr(), nb,
                                     stream) == sidm.OK
        assert np.array_equal(v1.cpu().numpy(), o["vel"]), call
        v2 = torch.from_numpy(vel).cuda()
        cnt = torch.zeros(p.n, dtype=torch.int32, device="cuda")
        assert ext.ext_apply_counting(rec_d.data_ptr(), rec.shape[0], v2.data_ptr(),
                                      mass_d.data_ptr(), cnt.data_ptr(), p.n, seed, step,
                                      scratch.data_ptr(), nb, stream) == sidm.OK
        assert np.array_equal(v2.cpu().numpy(), o["vel"]), call
        assert np.array_equal(cnt.cpu().numpy(), mult), call
        v3 = torch.from_numpy(vel).cuda()
        assert ext.ext_apply_builtin(rec_d.data_ptr(), rec.shape[0], v3.data_ptr(),
                                     mass_d.data_ptr(), p.n, seed, step, 1.0, scratch.data_ptr(),
                                     nb, stream) == sidm.OK
        assert np.array_equal(v3.cpu().numpy(), o["vel"]), call
        vel = o["vel"]


@pytest.mark.gpu
def test_builtin_inelastic_model_and_invalid_records(orc, ext):
    import torch
    p = I.uniform_box(8000, 1.0, 1.0, 93, ids="random")
    o, rec = _step_pairs(orc, p, 7, 3, inelastic=0.3)
    nb = ext.ext_scratch_bytes(p.n, rec.shape[0])
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    rec_d = torch.from_numpy(rec.view(np.uint8)).cuda()
    mass_d = torch.from_numpy(p.mass).cuda()
    v = torch.from_numpy(p.vel).cuda()
    st = ext.ext_apply_builtin(rec_d.data_ptr(), rec.shape[0], v.data_ptr(), mass_d.data_ptr(),
                               p.n, 7, 3, 0.7, scratch.data_ptr(), nb, None)
    assert st == sidm.OK
    assert np.array_equal(v.cpu().numpy(), o["vel"])
    bad = rec.copy()
    bad["ib"][5] = p.n                                 # outside [0, n): nothing is applied
    v = torch.from_numpy(p.vel).cuda()
    st = ext.ext_apply_elastic(torch.from_numpy(bad.view(np.uint8)).cuda().data_ptr(),
                               bad.shape[0], v.data_ptr(), mass_d.data_ptr(), p.n, 7, 3,
                               scratch.data_ptr(), nb, None)
    assert st == sidm.ERR_INVALID_ARG
    assert np.array_equal(v.cpu().numpy(), p.vel)
    # scratch too small
    st = ext.ext_apply_elastic(rec_d.data_ptr(), rec.shape[0], v.data_ptr(), mass_d.data_ptr(),
                               p.n, 7, 3, scratch.data_ptr(), nb - 256, None)
    assert st == sidm.ERR_INVALID_ARG
