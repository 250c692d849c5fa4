"""GPU check of the injectivity/dilation estimator (Fig. 2) against the oracle's exact eigenvalues.

With iters >= r the Lanczos tridiagonal holds the spectrum of S_r^T S_r, so alpha and beta must match
the oracle's dense eigenvalues to 1e-8 relative.  With fewer steps the estimates are Ritz values:
beta <= the true beta and alpha >= the true alpha, beta within 1e-3 and alpha within 10% after 300
steps at r = 3000.  The CSR and column draws are checked through these products.
"""
import numpy as np
import pytest
import torch

from oracle import osi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


@pytest.mark.parametrize("kind", ["stack", "uniform"])
@pytest.mark.parametrize("r,zeta", [(1, 4), (60, 4), (500, 8)])
def test_exact_with_full_lanczos(rsk, kind, r, zeta):
    k = max(2 * r, zeta) if kind == "uniform" else -(-max(2 * r, zeta) // zeta) * zeta
    a, b = rsk.rsk_osi_estimate(r, k=k, zeta=zeta, seed=4, kind=kind, iters=2 * r + 10)
    ao, bo = osi.extremes(r, k, zeta, 4, {"uniform": 0, "stack": 1}[kind])
    assert abs(a - ao) <= 1e-8 * max(1.0, ao) and abs(b - bo) <= 1e-8 * bo


def test_ritz_bounds_with_few_steps(rsk):
    r = 3000
    a, b = rsk.rsk_osi_estimate(r, zeta=8, seed=2, kind="stack", iters=300)
    ao, bo = osi.extremes(r, 2 * r, 8, 2, 1)
    assert b <= bo * (1 + 1e-12) and a >= ao * (1 - 1e-12)
    assert b >= bo * (1 - 1e-3) and a <= ao * 1.10
