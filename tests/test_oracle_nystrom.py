"""Pins of the Nystrom oracle (Alg. 2) against what the mathematics fixes.

* Without the shift, Alg. 2's U diag(Lambda) U^T equals the definition Y (Omega^T Y)^+ Y^T;
* a psd A of rank r < k is recovered exactly without the shift (the Nystrom approximation is exact
  on rank-r matrices when Omega^T Y has rank r) and to a small multiple of the shift with it;
* A - A_hat is psd (the Nystrom approximation never exceeds A), and ||A - A_hat||_2 is at least the
  best rank-k error lambda_{k+1}(A) (Eckart-Young);
* U has orthonormal columns and Lambda >= 0, descending.
"""
import numpy as np
import pytest

from oracle import nystrom as ony


def psd_matrix(n, decay, seed, rank=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = decay ** np.arange(n)
    if rank is not None:
        lam[rank:] = 0
    return (Q * lam) @ Q.T, lam


@pytest.mark.parametrize("kind", [0, 1])
def test_unshifted_equals_definition(kind):
    A, _ = psd_matrix(120, 0.9, 1)
    U, lam = ony.psd_nystrom(A, 24, 4, 7, kind=kind, eps=0.0)
    np.testing.assert_allclose((U * lam) @ U.T, ony.psd_nystrom_direct(A, 24, 4, 7, kind=kind), atol=1e-10)


@pytest.mark.parametrize("kind", [0, 1])
def test_low_rank_recovered(kind):
    A, _ = psd_matrix(200, 0.8, 2, rank=10)
    U, lam = ony.psd_nystrom(A, 32, 8, 3, kind=kind)
    Ahat = (U * lam) @ U.T
    # exact up to the shift: the error is a small multiple of nu = sqrt(n) eps ||Y||_F
    Y = A @ ony.test_matrix(200, 32, 8, 3, kind)
    nu = np.sqrt(200) * ony.EPS32 * np.linalg.norm(Y)
    assert np.linalg.norm(A - Ahat, 2) <= 100 * nu
    # and exact (to rounding) from the unshifted definition (whose Cholesky form would fail here:
    # Omega^T Y has rank 10 < k, which is what the shift is for)
    assert np.linalg.norm(A - ony.psd_nystrom_direct(A, 32, 8, 3, kind=kind), 2) <= 1e-10


@pytest.mark.parametrize("kind", [0, 1])
def test_never_exceeds_a_and_eckart_young(kind):
    A, lam_true = psd_matrix(150, 0.85, 3)
    k = 20
    U, lam = ony.psd_nystrom(A, k, 4, 11, kind=kind, eps=0.0)
    E = A - (U * lam) @ U.T
    assert np.linalg.eigvalsh(0.5 * (E + E.T)).min() >= -1e-10
    assert np.linalg.norm(E, 2) >= lam_true[k] * (1 - 1e-9)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-10)
    assert np.all(lam >= 0) and np.all(np.diff(lam) <= 1e-15)


def lowrank(n, d, r, seed, decay=0.7):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    V, _ = np.linalg.qr(rng.standard_normal((d, r)))
    return (U * decay ** np.arange(r)) @ V.T


@pytest.mark.parametrize("kind", [0, 1])
def test_generalized_forms_equal_definition(kind):
    # Algs. 4 and 5 both compute Y (Psi^T Y)^+ Psi^T A (the generalized Nystrom approximation)
    rng = np.random.default_rng(5)
    A = lowrank(300, 200, 40, 6) + 1e-3 * rng.standard_normal((300, 200))
    k, p = 24, 36
    ref = ony.gen_nystrom_direct(A, k, p, 4, 9, kind=kind)
    F, G, r = ony.gen_nystrom_outer(A, k, p, 4, 9, kind=kind, eps=0.0)
    U, s, V, r5 = ony.gen_nystrom_svd(A, k, p, 4, 9, kind=kind, eps=0.0)
    assert r == k and r5 == k
    np.testing.assert_allclose(F @ G.T, ref, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose((U * s) @ V.T, ref, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-10)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-10)


@pytest.mark.parametrize("kind", [0, 1])
def test_generalized_exact_on_low_rank(kind):
    A = lowrank(400, 250, 12, 7)
    F, G, r = ony.gen_nystrom_outer(A, 20, 32, 4, 3, kind=kind)
    U, s, V, _ = ony.gen_nystrom_svd(A, 20, 32, 4, 3, kind=kind)
    assert r == 12   # numerical rank found by the 5 eps sigma_1 cut
    assert np.linalg.norm(A - F @ G.T, 2) <= 1e-10 * np.linalg.norm(A, 2)
    assert np.linalg.norm(A - (U * s) @ V.T, 2) <= 1e-10 * np.linalg.norm(A, 2)
