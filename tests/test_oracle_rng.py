"""Pins of the oracle's random-number building blocks (not GPU)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    """Philox4x32-10 reproduces the published known-answer vectors."""
    out = O.philox4x32_10(row[0:4], row[4:6])
    assert [int(x) for x in out] == row[6:10]


def _words(n, tag=9):
    w = np.array([O.philox4x32_10([k, 3, 0, tag], [17, 0]) for k in range(n)], dtype=np.uint64)
    return w


def test_box_muller_is_standard_normal():
    """Box-Muller of Philox words: both outputs N(0,1) and uncorrelated (KS test)."""
    w = _words(20000)
    z = np.array([O.box_muller(int(a), int(b)) for a, b in w[:, :2]])
    for col in range(2):
        assert stats.kstest(z[:, col], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5.0 / math.sqrt(len(z))


def test_box_muller_extremes_finite():
    """u1 = (w0+1)/2^32 never reaches 0, so the radius stays finite."""
    for w0 in (0, 1, 0xFFFFFFFF):
        for w1 in (0, 0x80000000, 0xFFFFFFFF):
            z0, z1 = O.box_muller(w0, w1)
            assert math.isfinite(z0) and math.isfinite(z1)
    z0, z1 = O.box_muller(0xFFFFFFFF, 0)   # u1 = 1 exactly: radius 0
    assert z0 == 0.0 and z1 == 0.0


def test_random_axis_uniform_on_sphere():
    """Random SRD axes are unit vectors with E[n] = 0 and E[n n^T] = I/3."""
    w = _words(20000, tag=3)
    n = np.array([O.random_axis(int(a), int(b)) for a, b in w[:, :2]])
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-14)
    assert np.all(np.abs(n.mean(0)) < 5 * math.sqrt(1 / 3 / len(n)))
    np.testing.assert_allclose(n.T @ n / len(n), np.eye(3) / 3, atol=0.01)
    # n_z uniform on [-1,1): Archimedes' hat-box theorem for a uniform sphere
    assert stats.kstest(n[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4
