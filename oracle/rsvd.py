"""Randomized SVD with a sparse sign test matrix (paper Alg. 1, Sec. 2.1) plus power iterations.

Alg. 1: Y = A Omega, Q = orth(Y), B = Q^T A, [Uhat, Sigma, V] = svd_econ(B), U = Q Uhat.
The paper's Alg. 1 has no power iterations; the q subspace iterations used here re-orthonormalise
after every product (Q = orth(A^T Q); Q = orth(A Q)), the usual stable form of
Halko-Martinsson-Tropp's power scheme.

Omega (N x r) is a SparseUniform test matrix with zeta nonzeros per row (Def. SparseUniform),
i.e. Omega^T is the left sparse sign matrix of oracle.sparse_sign drawn from Philox stream 3.

spectral_error: ||A - Q Q^T A||_2 by power iterations on the residual operator, started from a
Philox-seeded vector (stream 9).
TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np

from . import sparse_sign
from .philox import words

STREAM_ERR = 9


def omega(N, r, zeta, seed):
    """Dense Omega (N x r) = (S from stream 3)^T with entries +-zeta^{-1/2}."""
    St = sparse_sign.matrix(N, r, zeta, seed, stream=sparse_sign.STREAM_RSVD)
    return np.asarray(St.T.todense()) / np.sqrt(zeta)


def orth(Y):
    """Orthonormal basis of range(Y) by Householder QR with diag(R) >= 0 (FP64)."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def range_finder(A, r, power_iters, zeta, seed):
    """Q after the sketch and q power iterations (FP64)."""
    A = np.asarray(A, dtype=np.float64)
    Om = omega(A.shape[1], r, zeta, seed)
    Q = orth(A @ Om)
    for _ in range(power_iters):
        Q = orth(A.T @ Q)
        Q = orth(A @ Q)
    return Q


def rsvd(A, r, power_iters, zeta, seed):
    """(U, s, Vt) of the rank-r approximation Q Q^T A (Alg. 1 with power iterations)."""
    A = np.asarray(A, dtype=np.float64)
    Q = range_finder(A, r, power_iters, zeta, seed)
    B = Q.T @ A
    Uh, s, Vt = np.linalg.svd(B, full_matrices=False)
    return Q @ Uh, s, Vt


def start_vector(n, seed):
    """Deterministic start vector in [-1, 1)^n from Philox stream 9."""
    w = words(seed, STREAM_ERR, np.arange(n, dtype=np.uint64), 0).astype(np.float64)
    return w / 2.0**31 - 1.0


def spectral_error(A, Q, iters=30, seed=0):
    """Power-method estimate of ||(I - Q Q^T) A||_2 (FP64)."""
    A = np.asarray(A, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    v = start_vector(A.shape[1], seed)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        y = A @ v
        y = y - Q @ (Q.T @ y)
        est = np.linalg.norm(y)
        if est == 0.0:
            return 0.0
        v = A.T @ y  # M^T y = A^T (I - QQ^T) y = A^T y because y is orthogonal to range(Q)
        v /= np.linalg.norm(v)
    return float(est)
