"""The method behind the device kick's divisions by the pair mass (Eqs.
12-13), checked on the host: a C copy of its steps (Markstein's correction
from the correctly rounded reciprocal, then the remainder check) against
the correctly rounded quotient x / M.  The check must keep no wrong
quotient and lose no right one; the device falls back to the division
whenever it rejects q."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path_factory.mktemp("kdc") / "kick_division_check")
    subprocess.run([cc, "-O2", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "kick_division_check.c"), "-lm"], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2])
def test_remainder_check_keeps_only_correctly_rounded_quotients(checker, seed):
    out = subprocess.run([checker, "3000000", str(seed)], check=True, capture_output=True,
                         text=True).stdout.split()
    wrong, fallback, kept_bad, lost = map(int, out)
    assert wrong == 0
    assert kept_bad == 0
    assert lost == 0
    # Markstein's corrected quotient was right on every case drawn, so the
    # division fallback is not needed for these values
    assert fallback == 0


def test_a_planted_error_in_the_check_is_caught(checker, tmp_path):
    # the check with the spacing taken one binade too wide (a plausible slip)
    # must keep wrong quotients; this guards the test itself
    src = open(os.path.join(HERE, "kick_division_check.c")).read()
    bad = src.replace("- 1076 -", "- 1075 -")
    assert bad != src
    path = tmp_path / "bad.c"
    path.write_text(bad)
    exe = str(tmp_path / "bad")
    subprocess.run([shutil.which("gcc") or "cc", "-O2", "-ffp-contract=off", "-o", exe,
                    str(path), "-lm"], check=True)
    out = subprocess.run([exe, "200000", "3"], check=True, capture_output=True,
                         text=True).stdout.split()
    assert int(out[2]) > 0
