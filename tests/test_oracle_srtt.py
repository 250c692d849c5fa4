"""Pins for the oracle's SRTT (CPU only): the WHT against scipy's Sylvester Hadamard matrix,
orthogonality of the unsubsampled transform, the popcount definition against the fast
transform, and the isotropy that the scaled restriction is chosen to give (Sec. 1.6)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import srtt


@pytest.mark.parametrize("m", [0, 1, 3, 6, 10])
def test_fwht_matches_hadamard(m):
    n = 1 << m
    rng = np.random.default_rng(m)
    X = rng.standard_normal((n, 3))
    assert np.allclose(srtt.fwht(X), sla.hadamard(n) @ X, atol=1e-10 * n)


def test_hadamard_orthogonal():
    n = 256
    H = srtt.fwht(np.eye(n))
    assert np.array_equal(H.T @ H, n * np.eye(n))
    i = np.arange(n)
    pc = np.array([[bin(a & b).count("1") & 1 for b in i] for a in i])
    assert np.array_equal(H, 1 - 2 * pc)


def test_full_transform_is_orthogonal():
    # d = n: Y = n^{-1/2} P H D A with P a permutation -> Y^T Y = A^T A
    n, k = 128, 4
    A = np.random.default_rng(1).standard_normal((n, k))
    Y = srtt.apply(A, n, seed=3)
    assert np.allclose(Y.T @ Y, A.T @ A, atol=1e-11)
    assert sorted(srtt.subsample(n, n, 3).tolist()) == list(range(n))


def test_n_equals_one():
    A = np.array([[2.5, -1.0]])
    Y = srtt.apply(A, 1, seed=0)
    D = srtt.diag_signs(1, 0)
    assert np.allclose(Y, D[0] * A)


def test_rows_definition_matches_fast_path():
    n, d, k = 512, 40, 3
    A = np.random.default_rng(2).standard_normal((n, k))
    Y = srtt.apply(A, d, seed=9)
    sel = [0, 5, 17, 39]
    assert np.allclose(srtt.apply_rows(A, sel, d, seed=9), Y[sel], atol=1e-12)


def test_subsample_distinct_uniform():
    n, d, trials = 64, 8, 4000
    cnt = np.zeros(n)
    for s in range(trials):
        P = srtt.subsample(n, d, s)
        assert len(set(P.tolist())) == d and P.min() >= 0 and P.max() < n
        cnt[P] += 1
    p = cnt / trials
    assert np.allclose(p, d / n, atol=5 * np.sqrt(d / n / trials))


def test_diag_signs_balanced():
    n = 1 << 16
    D = srtt.diag_signs(n, 4).astype(float)
    assert abs(D.mean()) < 4 / np.sqrt(n)
    assert abs((D[:-1] * D[1:]).mean()) < 4 / np.sqrt(n)
    assert abs((D[:-32] * D[32:]).mean()) < 4 / np.sqrt(n)


def test_isotropy_monte_carlo():
    # M = d^{-1/2} P H D: E[M^T M] = I
    n, d, trials = 16, 4, 4000
    acc = np.zeros((n, n))
    for s in range(trials):
        M = srtt.apply(np.eye(n), d, seed=s)
        acc += M.T @ M
    acc /= trials
    assert np.abs(acc - np.eye(n)).max() < 0.08
