"""The built-in kick spread over a group of eight lanes (IsotropicKick::
scatter_group, Sec. 4.1 kick of Eqs. 12-13), which the kick application
uses, against the one-lane prepared kick it replaces: bit-identical on
random pairs with masses, velocities and eps over wide ranges.  The probe
also reports the costs behind the design: on this GPU a warp's FP64
instructions do not overlap (each holds the FP64 unit for a fixed number of
cycles whatever the number of active lanes), so spreading a pair's FP64
operations over lanes shortens the kick.  tests/kick_probe.cu is compiled
here with nvcc."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2607_05504_b300 import build as B

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    so = os.path.join(str(tmp_path_factory.mktemp("kick")), "libkick_probe.so")
    subprocess.check_call([B.NVCC, *B.ARCH, "-O3", "-std=c++17", "-fmad=false", "-shared",
                           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                           os.path.join(HERE, "kick_probe.cu"), "-o", so])
    L = C.CDLL(so)
    L.probe_group_differing.argtypes = [C.c_uint64, C.c_uint32, C.POINTER(C.c_ulonglong)]
    L.probe_cycles.argtypes = [C.POINTER(C.c_longlong)]
    return L


@pytest.mark.parametrize("seed", [1, 2])
def test_group_kick_is_bit_identical_to_the_one_lane_kick(probe, seed):
    bad = C.c_ulonglong(0)
    assert probe.probe_group_differing(1 << 23, seed, C.byref(bad)) == 0
    assert bad.value == 0


def test_group_kick_is_shorter_and_fp64_does_not_overlap(probe):
    out = (C.c_longlong * 6)()
    assert probe.probe_cycles(out) == 0
    dfma, two, ffma, dsqrt, one_lane, group = list(out)
    print(f"cycles: dependent FP64 FMA {dfma}, two independent {two}, FP32 FMA {ffma}, "
          f"dsqrt {dsqrt}, prepared kick on one lane {one_lane}, on a group of eight {group}")
    assert dfma > 4 * ffma
    assert two > 1.5 * dfma          # a warp's FP64 instructions do not overlap
    assert group < 0.9 * one_lane
