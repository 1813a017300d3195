"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point declared in include/sidm.h, and
rejects invalid configurations before touching a device."""
import ctypes as C
import os
import re

import pytest

from paper_2607_05504_b300 import build, sidm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sidm.h")).read()
    return sorted(set(re.findall(r"SIDM_API\s+[\w\s\*]+?\b(sidm_\w+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert set(_declared()) == set(sidm.ENTRY_POINTS)


def test_library_loads_and_exports_every_declared_symbol():
    L = sidm.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert os.path.dirname(sidm.lib_path()).endswith("paper_2607_05504_b300")


def test_error_strings():
    for st in (0, 1, 2, 4, -1, -2, -3, -4, -5):
        assert sidm.error_string(st)
    assert "unknown" in sidm.error_string(-99)


def test_default_config_is_the_papers_fiducial():
    c = sidm.sidm_default_config()
    assert (c.n_ngb, c.ngb_tol, c.c_sidm, c.kernel, c.precision) == (32, 5, 0.1, 0, 0)
    assert c.box == 0.0 and c.fixed_h == 0.0 and c.device == -1 and c.profile == 0


@pytest.mark.parametrize("field,value", [("n_ngb", 0), ("ngb_tol", -1), ("ngb_tol", 32),
                                         ("c_sidm", 0.0), ("box", -1.0), ("kernel", 7),
                                         ("precision", 3), ("fixed_h", -1.0), ("n_max", -5),
                                         ("n_ngb", 300),
                                         # K + 1 = n_ngb + tol + 2 must stay <= 256
                                         ("n_ngb", 250),
                                         ("max_resolver_passes", -1), ("rebuild_every", -1),
                                         ("pair_capacity", -1), ("estimator", 5),
                                         ("box", float("inf")), ("fixed_h", float("nan"))])
def test_create_rejects_invalid_config(field, value):
    c = sidm.sidm_default_config()
    setattr(c, field, value)
    h = C.c_void_p()
    assert sidm.lib().sidm_create(C.byref(c), C.byref(h)) == sidm.ERR_INVALID_ARG
    assert not h.value


def test_null_arguments_are_rejected():
    L = sidm.lib()
    assert L.sidm_create(None, None) == sidm.ERR_INVALID_ARG
    assert L.sidm_step(None, None, None, 1.0, None, 0, None) == sidm.ERR_INVALID_ARG
    assert L.sidm_sync(None) == sidm.ERR_INVALID_ARG
    assert L.sidm_kernel_launches(None) == -1


def test_build_is_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert "-fmad=false" in build.FLAGS
