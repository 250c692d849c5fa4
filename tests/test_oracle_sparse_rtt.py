"""Pins of the SparseRTT oracle (Def. SparseRTT, Def. SparseCol) against what the definitions fix.

* the fast form equals Omega^T A with Omega = D F S built densely from the definitions: D the
  Rademacher diagonal, F = H_n / sqrt(n) from scipy's Hadamard matrix, S the SparseCol matrix with
  columns d^{-1/2} sqrt(n/xi) sum_t rho_t e_{s_t};
* every column of S has xi distinct positions and squared norm n/d exactly;
* isotropy E[Omega Omega^T] = I (the first moment E[W] = k^{-1} I of the SparseCol moment lemma,
  summed over the columns), by Monte Carlo over seeds;
* with xi = n every column of S holds every coordinate once (a signed all-ones pattern).
"""
import numpy as np
from scipy.linalg import hadamard

from oracle import srtt as osr


def dense_omega(n, d, xi, seed):
    D = np.diag(osr.diag_signs(n, seed).astype(np.float64))
    F = hadamard(n).astype(np.float64) / np.sqrt(n)
    pos, sg = osr.sparse_rtt_positions(n, d, xi, seed)
    S = np.zeros((n, d))
    for q in range(d):
        for t in range(xi):
            S[pos[q, t], q] += sg[q, t] * np.sqrt(n / xi) / np.sqrt(d)
    return D @ F @ S, S


def test_fast_form_equals_dense_definition():
    rng = np.random.default_rng(0)
    for n, d, xi, seed in [(8, 3, 2, 1), (64, 20, 5, 2), (256, 40, 9, 3)]:
        A = rng.standard_normal((n, 4))
        Omega, _ = dense_omega(n, d, xi, seed)
        np.testing.assert_allclose(osr.sparse_rtt_apply(A, d, xi, seed), Omega.T @ A, rtol=0, atol=1e-12)


def test_columns_distinct_and_norm():
    n, d, xi = 128, 50, 7
    pos, sg = osr.sparse_rtt_positions(n, d, xi, seed=4)
    for q in range(d):
        assert len(set(pos[q].tolist())) == xi
    assert pos.min() >= 0 and pos.max() < n and set(np.unique(sg)) <= {-1, 1}
    _, S = dense_omega(n, d, xi, seed=4)
    np.testing.assert_allclose((S * S).sum(axis=0), n / d, rtol=1e-14)


def test_isotropy_monte_carlo():
    n, d, xi, trials = 16, 8, 3, 2000
    G = np.zeros((n, n))
    for t in range(trials):
        Omega, _ = dense_omega(n, d, xi, seed=500 + t)
        G += Omega @ Omega.T
    G /= trials
    assert np.abs(G - np.eye(n)).max() < 0.1


def test_full_column_sparsity():
    n, d = 16, 5
    pos, sg = osr.sparse_rtt_positions(n, d, n, seed=7)
    for q in range(d):
        assert sorted(pos[q].tolist()) == list(range(n))
