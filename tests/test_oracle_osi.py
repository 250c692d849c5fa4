"""Pins of the injectivity/dilation oracle (Fig. 2).

* the columns of S have unit norm, so trace(S_r^T S_r) = r and alpha <= 1 <= beta exactly;
* r = 1 gives alpha = beta = 1;
* for SparseStack with zeta = 8 and k = 2r the estimates sit near the Gaussian asymptotes
  (1 -+ 1/sqrt(2))^2 that the figure marks (within 25% at r = 400).
"""
import numpy as np
import pytest

from oracle import osi


@pytest.mark.parametrize("kind", [0, 1])
def test_trace_and_order(kind):
    S = osi.first_columns(50, 96, 8, 3, kind)
    G = S.T @ S
    assert abs(np.trace(G) - 50) <= 1e-12
    a, b = osi.extremes(50, 96, 8, 3, kind)
    assert a <= 1 + 1e-12 and b >= 1 - 1e-12


@pytest.mark.parametrize("kind", [0, 1])
def test_single_column(kind):
    a, b = osi.extremes(1, 16, 4, 0, kind)
    assert abs(a - 1) <= 1e-14 and abs(b - 1) <= 1e-14


def test_stack_near_gaussian_asymptotes():
    r = 400
    a, b = osi.extremes(r, 2 * r, 8, 1, kind=1)
    ga, gb = (1 - 1 / np.sqrt(2)) ** 2, (1 + 1 / np.sqrt(2)) ** 2
    assert abs(a - ga) <= 0.25 * ga
    assert abs(b - gb) <= 0.25 * gb
