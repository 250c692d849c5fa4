"""SparseUniform sparse sign embedding: generation, inverted index and the sketch S @ A.

Paper: Def. "SparseUniform" (Sec. 3.2.1): exactly zeta entries zeta^{-1/2} * rho per row of
the right test matrix Omega, at positions drawn uniformly without replacement, rho
Rademacher.  The left sketch S = Psi^T used here is the transpose: S is d x n with exactly
zeta nonzeros per *column*.  The sketch application Psi^T A costs O(zeta nnz(A))
(Sec. 1.5, SparseStack cost discussion; Sec. 3.2).

Readings of what the paper leaves open (both sides implement the same rule):
  * Sampling without replacement is Floyd's algorithm (Bentley & Floyd, CACM 1987) fed by
    the Philox stream ``stream`` (0 for the left sketch), entity = column j:
        for q = 0..zeta-1:  m = d - zeta + q;  t = floor(w_q * (m + 1) / 2^32)
                            chosen_q = m if t already chosen else t
    where w_q = word(seed, stream, j, q).
  * The sign of the q-th chosen row is bit q of w_zeta (set bit = -1), so zeta <= 32.
  * The scale zeta^{-1/2} is applied once to the +-1 weighted sums.

TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np
import scipy.sparse as sp

from .philox import words

STREAM_LEFT = 0
STREAM_RSVD = 3


def columns(n, d, zeta, seed, stream=STREAM_LEFT, col0=0):
    """Rows (n x zeta, int64, insertion order) and signs (n x zeta, int8 in {+1,-1}) of the
    columns col0 .. col0 + n - 1 of S.

    Row q of column j is the q-th index Floyd's algorithm inserts.
    """
    if not (1 <= zeta <= 32 and zeta <= d):
        raise ValueError("need 1 <= zeta <= min(d, 32)")
    j = np.arange(col0, col0 + n, dtype=np.uint64)
    rows = np.empty((n, zeta), dtype=np.int64)
    for q in range(zeta):
        w = words(seed, stream, j, q).astype(np.uint64)
        m = d - zeta + q
        t = ((w * np.uint64(m + 1)) >> np.uint64(32)).astype(np.int64)
        dup = np.zeros(n, dtype=bool)
        for p in range(q):
            dup |= rows[:, p] == t
        rows[:, q] = np.where(dup, m, t)
    sbits = words(seed, stream, j, zeta).astype(np.int64)
    q = np.arange(zeta, dtype=np.int64)
    signs = np.where((sbits[:, None] >> q[None, :]) & 1, -1, 1).astype(np.int8)
    return rows, signs


def sign_bits(signs):
    """Pack a (n x zeta) +-1 array into one uint32 per column (bit q set = -1)."""
    n, zeta = signs.shape
    out = np.zeros(n, dtype=np.uint64)
    for q in range(zeta):
        out |= (signs[:, q] < 0).astype(np.uint64) << np.uint64(q)
    return out.astype(np.uint32)


def dense(n, d, zeta, seed, stream=STREAM_LEFT):
    """The d x n matrix S with entries in {0, +-zeta^{-1/2}} (tiny sizes only)."""
    rows, signs = columns(n, d, zeta, seed, stream)
    S = np.zeros((d, n), dtype=np.float64)
    for j in range(n):
        for q in range(zeta):
            S[rows[j, q], j] = signs[j, q] / np.sqrt(zeta)
    return S


def csr(n, d, zeta, seed, stream=STREAM_LEFT):
    """Inverted index of S: row i lists the columns j with S[i, j] != 0 in ascending j.

    Returns (rowptr[d+1], cols[n*zeta], negative[n*zeta]) with int64 / bool arrays.
    """
    rows, signs = columns(n, d, zeta, seed, stream)
    r = rows.reshape(-1)
    j = np.repeat(np.arange(n, dtype=np.int64), zeta)
    neg = (signs.reshape(-1) < 0)
    order = np.lexsort((j, r))  # primary key: row r, secondary: column j
    counts = np.bincount(r, minlength=d)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, j[order], neg[order]


def matrix(n, d, zeta, seed, stream=STREAM_LEFT):
    """S as a scipy CSR matrix (d x n) with the +-1 pattern (unscaled)."""
    rows, signs = columns(n, d, zeta, seed, stream)
    jj = np.repeat(np.arange(n), zeta)
    return sp.csr_matrix((signs.reshape(-1).astype(np.float64), (rows.reshape(-1), jj)), shape=(d, n))


def apply(A, d, zeta, seed, stream=STREAM_LEFT):
    """SA = zeta^{-1/2} * (S~ @ A) in float64, S~ the +-1 pattern.  A is n x k."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    St = matrix(n, d, zeta, seed, stream)
    return np.asarray(St @ A) / np.sqrt(zeta)


def abs_apply(A, d, zeta, seed, stream=STREAM_LEFT):
    """(|S~| @ |A|) in float64, the elementwise scale that bounds summation error."""
    A = np.abs(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    St = abs(matrix(n, d, zeta, seed, stream))
    return np.asarray(St @ A)


def apply_block(A_block, col0, d, zeta, seed, stream=STREAM_LEFT):
    """zeta^{-1/2} * S~[:, col0:col0+nb] @ A_block: the part of S A that rows col0 .. col0+nb-1 of
    a row-partitioned A contribute (S A is the sum of these over the blocks of any partition)."""
    A_block = np.asarray(A_block, dtype=np.float64)
    nb = A_block.shape[0]
    rows, signs = columns(nb, d, zeta, seed, stream, col0=col0)
    jj = np.repeat(np.arange(nb), zeta)
    St = sp.csr_matrix((signs.reshape(-1).astype(np.float64), (rows.reshape(-1), jj)), shape=(d, nb))
    return np.asarray(St @ A_block) / np.sqrt(zeta)


def abs_apply_block(A_block, col0, d, zeta, seed, stream=STREAM_LEFT):
    """(|S~[:, col0:col0+nb]| @ |A_block|) in float64: abs_apply for a row block."""
    A_block = np.abs(np.asarray(A_block, dtype=np.float64))
    nb = A_block.shape[0]
    rows, _ = columns(nb, d, zeta, seed, stream, col0=col0)
    jj = np.repeat(np.arange(nb), zeta)
    St = sp.csr_matrix((np.ones(nb * zeta), (rows.reshape(-1), jj)), shape=(d, nb))
    return np.asarray(St @ A_block)
