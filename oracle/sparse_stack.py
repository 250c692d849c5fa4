"""SparseStack test matrix: a stack of zeta independent CountSketches, and the sketch S @ A.

Paper: Def. SparseStack (Sec. 1.5): with block size b and row sparsity zeta, the test matrix
Omega (ambient x k, k = b * zeta) has in each row zeta entries zeta^{-1/2} * rho_{iq} e_{s_iq}^T,
one in each of the zeta column blocks of width b, with s_iq uniform on {1..b} and rho_iq
Rademacher, all independent.  As in the SparseUniform oracle the left sketch is S = Omega^T
(d x n, d = b * zeta), so every column j of S has one nonzero in each block of b consecutive rows.

Reading (both sides implement the same rule): the draws of column j are w_q = word(seed, 4, j, q)
(Philox stream 4); the row in block q is q*b + floor(w_q * b / 2^32); the sign of that entry is
bit q of w_zeta (set bit = -1).  The scale zeta^{-1/2} is applied once to the +-1 sums.

TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np
import scipy.sparse as sp

from .philox import words

STREAM_STACK = 4


def columns(n, d, zeta, seed, stream=STREAM_STACK):
    """Rows (n x zeta, int64; entry q lies in block q) and signs (n x zeta, int8 +-1) of S."""
    if not (1 <= zeta <= 32 and zeta <= d and d % zeta == 0):
        raise ValueError("need 1 <= zeta <= min(d, 32) and d a multiple of zeta")
    b = d // zeta
    j = np.arange(n, dtype=np.uint64)
    rows = np.empty((n, zeta), dtype=np.int64)
    for q in range(zeta):
        w = words(seed, stream, j, q).astype(np.uint64)
        rows[:, q] = q * b + ((w * np.uint64(b)) >> np.uint64(32)).astype(np.int64)
    sbits = words(seed, stream, j, zeta).astype(np.int64)
    q = np.arange(zeta, dtype=np.int64)
    signs = np.where((sbits[:, None] >> q[None, :]) & 1, -1, 1).astype(np.int8)
    return rows, signs


def dense(n, d, zeta, seed):
    """The d x n matrix S with entries in {0, +-zeta^{-1/2}} (tiny sizes only)."""
    rows, signs = columns(n, d, zeta, seed)
    S = np.zeros((d, n), dtype=np.float64)
    for j in range(n):
        for q in range(zeta):
            S[rows[j, q], j] = signs[j, q] / np.sqrt(zeta)
    return S


def matrix(n, d, zeta, seed):
    """S as a scipy CSR matrix (d x n) with the +-1 pattern (unscaled)."""
    rows, signs = columns(n, d, zeta, seed)
    jj = np.repeat(np.arange(n), zeta)
    return sp.csr_matrix((signs.reshape(-1).astype(np.float64), (rows.reshape(-1), jj)), shape=(d, n))


def apply(A, d, zeta, seed):
    """SA = zeta^{-1/2} * (S~ @ A) in float64 (A is n x k)."""
    A = np.asarray(A, dtype=np.float64)
    return np.asarray(matrix(A.shape[0], d, zeta, seed) @ A) / np.sqrt(zeta)


def abs_apply(A, d, zeta, seed):
    """(|S~| @ |A|) in float64."""
    A = np.abs(np.asarray(A, dtype=np.float64))
    return np.asarray(abs(matrix(A.shape[0], d, zeta, seed)) @ A)
