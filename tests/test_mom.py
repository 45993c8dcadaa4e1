"""The (epsilon, delta) amplification's host logic (library functions that
need no GPU): median of group means and the sizes, against closed cases and
the two inequalities the sizes are chosen to meet."""
import math

import numpy as np
import pytest

from paper_1801_00338_gb300 import bfc
from paper_1801_00338_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return bfc.load()


def test_median_of_means_closed_cases(lib):
    y = np.arange(1, 13, dtype=np.float64)          # 1..12
    assert bfc.bfc_median_of_means(y, 1) == pytest.approx(6.5)          # one group: the mean
    assert bfc.bfc_median_of_means(y, 12) == pytest.approx(6.5)         # singleton groups: the median
    assert bfc.bfc_median_of_means(y[:11], 11) == 6.0                   # odd count: the middle value
    # groups of 4: means 2.5, 6.5, 10.5 -> 6.5; groups of 3: 2, 5, 8, 11 -> (5 + 8) / 2
    assert bfc.bfc_median_of_means(y, 3) == pytest.approx(6.5)
    assert bfc.bfc_median_of_means(y, 4) == pytest.approx(6.5)
    # an outlying group cannot move the median
    z = np.array([1.0, 1.0, 1.0, 1.0, 1e12, 1e12], np.float64)
    assert bfc.bfc_median_of_means(z, 3) == pytest.approx(1.0)
    assert bfc.bfc_median_of_means(np.full(10, 7.25), 5) == 7.25


def test_median_of_means_rejects_bad_sizes(lib):
    y = np.ones(10)
    for g in (0, 3, 20):
        with pytest.raises(bfc.BfcError):
            bfc.bfc_median_of_means(y, g)
    with pytest.raises(bfc.BfcError):
        bfc.bfc_median_of_means(np.ones(0), 1)


@pytest.mark.parametrize("var1,Bv,eps,delta", [(1e6, 100.0, 0.1, 0.05), (4.8e26, 1.5e11, 0.01, 0.01),
                                               (0.0, 5.0, 0.5, 0.5), (2.0, 1.0, 0.2, 1e-6)])
def test_sizes_meet_their_inequalities(lib, var1, Bv, eps, delta):
    alpha, g = bfc.bfc_mom_sizes(var1, Bv, eps, delta)
    # Chebyshev: Var / (alpha eps^2 B^2) <= 1/32, and alpha is the least such count
    assert var1 / (alpha * eps * eps * Bv * Bv) <= 1 / 32 * (1 + 1e-12)
    assert alpha == 1 or var1 / ((alpha - 1) * eps * eps * Bv * Bv) > 1 / 32
    # Hoeffding: at least half of g groups miss with probability <= exp(-2 g (1/2 - 1/32)^2) <= delta
    assert g % 2 == 1
    assert math.exp(-2 * g * (0.5 - 1 / 32) ** 2) <= delta
    assert g <= 2 or math.exp(-2 * (g - 2) * (0.5 - 1 / 32) ** 2) > delta


def test_sizes_reject_bad_arguments(lib):
    for args in ((-1.0, 1.0, 0.1, 0.1), (1.0, 0.0, 0.1, 0.1), (1.0, 1.0, 0.0, 0.1), (1.0, 1.0, 0.1, 1.0),
                 (1.0, 1.0, 0.1, 0.0), (1e40, 1.0, 1e-9, 0.1)):
        with pytest.raises(bfc.BfcError):
            bfc.bfc_mom_sizes(*args)
