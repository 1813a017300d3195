"""The library's table of the kernel-overlap estimator (its own quadrature:
spherical shells with the angular integral in closed form) against the
oracle's independent cylindrical quadrature, and the table validation of the
host entry point.  Host only: no GPU call."""
import numpy as np
import pytest

import oracle
from paper_2607_05504_b300 import sidm


@pytest.mark.parametrize("kernel", [0, 1])
def test_library_table_matches_the_oracle_quadrature(kernel):
    a = sidm.sidm_overlap_table(kernel, 24, 96)
    b = oracle.overlap_table(24, 96, kernel=kernel)
    assert a.shape == b.shape == (25, 97)
    assert np.max(np.abs(a - b)) < 2e-9 * np.max(b)
    assert np.all(a >= 0.0) and np.all(a[:, -1] == 0.0)


def test_library_table_rejects_bad_shapes():
    with pytest.raises(sidm.SidmError):
        sidm.sidm_overlap_table(0, 0, 10)
    with pytest.raises(sidm.SidmError):
        sidm.sidm_overlap_table(2, 4, 10)
