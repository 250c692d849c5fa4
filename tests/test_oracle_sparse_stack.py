"""Pins of the SparseStack oracle (Def. SparseStack) against what the definition fixes.

* structure: every column has exactly one nonzero of magnitude zeta^{-1/2} in each block of b rows;
* the row inside a block is uniform on the b rows (chi-square over many columns);
* every column has unit norm, so diag(S^T S) = 1 exactly for every draw;
* isotropy E[S^T S] = I (the CountSketch moment E[Phi Phi^T] = I of the paper's lemma on
  CountSketch moments, averaged over the zeta blocks), and E[S S^T] = (n/d) I, by Monte Carlo;
* a brute-force dense product equals the sparse apply.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import sparse_stack as ost


def test_one_entry_per_block():
    n, d, zeta = 500, 48, 6
    rows, signs = ost.columns(n, d, zeta, seed=3)
    b = d // zeta
    assert np.array_equal(rows // b, np.broadcast_to(np.arange(zeta), rows.shape))
    assert set(np.unique(signs)) <= {-1, 1}
    S = ost.dense(n, d, zeta, seed=3)
    assert np.all(np.count_nonzero(S, axis=0) == zeta)
    np.testing.assert_allclose(np.abs(S[S != 0]), 1 / np.sqrt(zeta))
    np.testing.assert_allclose((S * S).sum(axis=0), 1.0, rtol=0, atol=1e-15)


def test_rows_uniform_within_block():
    n, d, zeta = 40_000, 20, 4
    rows, signs = ost.columns(n, d, zeta, seed=8)
    b = d // zeta
    for q in range(zeta):
        counts = np.bincount(rows[:, q] - q * b, minlength=b)
        assert stats.chisquare(counts).pvalue > 1e-4
    # balanced, independent signs
    assert abs(signs.mean()) < 0.02


def test_isotropy_monte_carlo():
    n, d, zeta, trials = 12, 16, 4, 3000
    G = np.zeros((n, n))
    H = np.zeros((d, d))
    for t in range(trials):
        S = ost.dense(n, d, zeta, seed=100 + t)
        G += S.T @ S
        H += S @ S.T
    G /= trials
    H /= trials
    assert np.abs(G - np.eye(n)).max() < 0.08
    assert np.abs(H - (n / d) * np.eye(d)).max() < 0.08
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-12)


def test_dense_product_equals_sparse_apply():
    rng = np.random.default_rng(2)
    n, d, zeta = 300, 40, 8
    A = rng.standard_normal((n, 5))
    np.testing.assert_allclose(ost.apply(A, d, zeta, 9), ost.dense(n, d, zeta, 9) @ A, rtol=0, atol=1e-13)


def test_rejects_d_not_multiple_of_zeta():
    with pytest.raises(ValueError):
        ost.columns(10, 30, 8, 0)
