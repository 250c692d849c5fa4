"""Randomized Nystrom approximations with structured sketching.

Paper: Alg. 2 (Sec. 2.2, Nystrom approximation of a psd matrix with a shift) and Algs. 4 and 5
(Sec. 2.4, generalized Nystrom in outer-product and SVD form).  Plain FP64 numpy/scipy,
written from the algorithms' steps in the paper's order.

Readings (both sides implement them):
  * The test matrices are the left sparse sketches of the other oracle modules transposed:
    Omega = S^T with S SparseUniform (kind 0) or SparseStack (kind 1), zeta nonzeros per row of
    Omega; Psi (Algs. 4/5) is drawn like Omega from seed + 1.
  * Alg. 2's shift nu = sqrt(n) eps ||Y|| uses eps = 2^-24 (the library computes in FP32) and the
    Frobenius norm of Y (an upper bound of the spectral norm, so the shift is never smaller).
  * Algs. 4/5's numerical-rank cut keeps singular values above 5 eps sigma_1 with eps = 2^-24.

TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np
import scipy.linalg as sla

from . import sparse_sign as _ss
from . import sparse_stack as _st

EPS32 = 2.0 ** -24


def test_matrix(n, k, zeta, seed, kind):
    """Omega (n x k, dense) = S^T for the k x n sparse sketch S of the given kind."""
    if kind == 1:
        S = _st.dense(n, k, zeta, seed)
    else:
        S = _ss.dense(n, k, zeta, seed)
    return S.T


def psd_nystrom(A, k, zeta, seed, kind=1, rank=None, eps=EPS32):
    """Alg. 2: U (n x rank, orthonormal) and Lambda (rank, descending, >= 0) with A ~ U diag(Lambda) U^T."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    rank = k if rank is None else rank
    Om = test_matrix(n, k, zeta, seed, kind)
    Y = A @ Om
    nu = np.sqrt(n) * eps * np.linalg.norm(Y)
    Ynu = Y + nu * Om
    M = Om.T @ Ynu
    C = np.linalg.cholesky(0.5 * (M + M.T)).T          # upper: M = C^T C
    B = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T   # B = Y_nu C^{-1}
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    lam = np.maximum(0.0, s ** 2 - nu)
    return U[:, :rank], lam[:rank]


def psd_nystrom_direct(A, k, zeta, seed, kind=1):
    """The Nystrom approximation Y (Omega^T Y)^+ Y^T from its definition (no shift), for pins."""
    A = np.asarray(A, dtype=np.float64)
    Om = test_matrix(A.shape[0], k, zeta, seed, kind)
    Y = A @ Om
    return Y @ np.linalg.pinv(Om.T @ Y) @ Y.T


def gen_nystrom_sketches(A, k, p, zeta, seed, kind=1):
    """Y = A Omega (n x k) and X = A^T Psi (d x p): Omega = S^T of a k x d sketch (seed), Psi = S'^T of
    a p x n sketch (seed + 1)."""
    A = np.asarray(A, dtype=np.float64)
    n, d = A.shape
    Om = test_matrix(d, k, zeta, seed, kind)
    Psi = test_matrix(n, p, zeta, seed + 1, kind)
    return A @ Om, A.T @ Psi, Om, Psi


def numerical_rank(s, eps=EPS32):
    return int(np.sum(s > 5 * eps * s[0])) if s.size and s[0] > 0 else 0


def gen_nystrom_outer(A, k, p, zeta, seed, kind=1, eps=EPS32):
    """Alg. 4: F (n x r), G (d x r) with A ~ F G^T, and the numerical rank r."""
    Y, X, Om, _ = gen_nystrom_sketches(A, k, p, zeta, seed, kind)
    U, s, Vt = np.linalg.svd(X.T @ Om, full_matrices=False)
    r = numerical_rank(s, eps)
    F = Y @ Vt[:r].T / s[:r]
    G = X @ U[:, :r]
    return F, G, r


def gen_nystrom_svd(A, k, p, zeta, seed, kind=1, eps=EPS32):
    """Alg. 5: U (n x k), sigma (k), V (d x k) with A ~ U diag(sigma) V^T, and the numerical rank r."""
    Y, X, Om, Psi = gen_nystrom_sketches(A, k, p, zeta, seed, kind)
    Q, _ = np.linalg.qr(Y)
    P, T = np.linalg.qr(X)
    U1, s1, V1t = np.linalg.svd(Psi.T @ Q, full_matrices=False)
    r = numerical_rank(s1, eps)
    C = V1t[:r].T @ ((U1[:, :r].T @ T.T) / s1[:r, None])
    Uh, s, Vht = np.linalg.svd(C, full_matrices=False)
    return Q @ Uh, s, P @ Vht.T, r


def gen_nystrom_direct(A, k, p, zeta, seed, kind=1):
    """The generalized Nystrom approximation Y (Psi^T Y)^+ Psi^T A from its definition (for pins)."""
    A = np.asarray(A, dtype=np.float64)
    Y, X, _, Psi = gen_nystrom_sketches(A, k, p, zeta, seed, kind)
    return Y @ np.linalg.pinv(Psi.T @ Y) @ X.T
