"""Subsampled randomized trigonometric transform with the Walsh-Hadamard transform.

Paper: the transform template Omega = D F S (Sec. 1.6, Eq. "intro-srtt"): D diagonal with iid
Rademacher entries, F a unitary trigonometric transform (here the WHT), and S a scaled
restriction that keeps k coordinates chosen uniformly at random so that Omega is isotropic.
The paper's cost accounting (Sec. 4.x "Arithmetic costs", steps 1-3) is y1 = D x,
y2 = F y1 (fast transform), y = S^T y2.

As a left sketch of a tall n x k matrix A with output dimension d this is
    Y = sqrt(n/d) * P * (H_n / sqrt(n)) * D * A = d^{-1/2} * P * H_n * D * A,
with H_n[i, l] = (-1)^{popcount(i & l)} (Sylvester / natural order), n = 2^m.

Readings (both sides): D_i = -1 iff bit (i & 31) of word(seed, 1, i >> 7, (i >> 5) & 3) is
set; P is Floyd's algorithm over [0, n) with d draws w_q = word(seed, 2, 0, q), output row q
being the q-th inserted coordinate; Sylvester ordering for H.

TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np

from .philox import words
from . import sparse_sign as _ss

STREAM_D = 1
STREAM_P = 2
STREAM_SPARSECOL = 5


def diag_signs(n, seed):
    """Rademacher diagonal D as an int8 vector of +-1."""
    i = np.arange(n, dtype=np.uint64)
    w = words(seed, STREAM_D, i >> np.uint64(7), (i >> np.uint64(5)) & np.uint64(3)).astype(np.uint64)
    bit = (w >> (i & np.uint64(31))) & np.uint64(1)
    return np.where(bit == 1, -1, 1).astype(np.int8)


def subsample(n, d, seed):
    """d distinct coordinates of [0, n) in Floyd insertion order (int64)."""
    if not 1 <= d <= n:
        raise ValueError("need 1 <= d <= n")
    q = np.arange(d, dtype=np.uint64)
    w = words(seed, STREAM_P, np.zeros(d, dtype=np.uint64), q).astype(np.uint64)
    chosen = set()
    out = np.empty(d, dtype=np.int64)
    for qq in range(d):
        m = n - d + qq
        t = int((int(w[qq]) * (m + 1)) >> 32)
        v = m if t in chosen else t
        chosen.add(v)
        out[qq] = v
    return out


def fwht(X):
    """Unnormalised Walsh-Hadamard transform along axis 0, Sylvester order (returns H @ X)."""
    Y = np.array(X, dtype=np.float64, copy=True)
    n = Y.shape[0]
    if n & (n - 1):
        raise ValueError("n must be a power of two")
    h = 1
    while h < n:
        Y = Y.reshape(n // (2 * h), 2, h, *Y.shape[1:])
        a = Y[:, 0].copy()
        b = Y[:, 1].copy()
        Y[:, 0] = a + b
        Y[:, 1] = a - b
        Y = Y.reshape(n, *Y.shape[3:])
        h *= 2
    return Y


def apply(A, d, seed):
    """Y = d^{-1/2} * (H_n D A)[P, :] in float64 for A of shape n x k (n a power of two)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    D = diag_signs(n, seed).astype(np.float64)
    HDA = fwht(D[:, None] * A.reshape(n, -1))
    P = subsample(n, d, seed)
    return HDA[P] / np.sqrt(d)


def apply_rows(A, rows_q, d, seed):
    """Selected output rows of the SRTT computed one by one from the definition.

    Y[q, :] = d^{-1/2} * sum_i (-1)^{popcount(P_q & i)} D_i A[i, :] for each q in rows_q.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    D = diag_signs(n, seed).astype(np.float64)
    P = subsample(n, d, seed)
    i = np.arange(n, dtype=np.int64)
    out = []
    for q in rows_q:
        x = P[q] & i
        par = np.zeros(n, dtype=np.int64)
        while np.any(x):
            par ^= x & 1
            x >>= 1
        h = 1.0 - 2.0 * par
        out.append((h * D) @ A / np.sqrt(d))
    return np.stack(out)


def apply_block(A_block, row0, n, d, seed):
    """The part of the n-row SRTT that rows row0 .. row0 + nb - 1 contribute, from the definition:
    Y_block[q, :] = d^{-1/2} * sum_{i in block} (-1)^{popcount(P_q & i)} D_i A[i, :].  The SRTT of A
    is the sum of these over the blocks of any row partition."""
    A_block = np.asarray(A_block, dtype=np.float64)
    nb = A_block.shape[0]
    if row0 < 0 or row0 + nb > n:
        raise ValueError("block outside [0, n)")
    D = diag_signs(n, seed)[row0:row0 + nb].astype(np.float64)
    P = subsample(n, d, seed)
    x = P[:, None] & np.arange(row0, row0 + nb, dtype=np.int64)[None, :]
    par = np.zeros_like(x)
    while np.any(x):
        par ^= x & 1
        x >>= 1
    H = 1.0 - 2.0 * par
    return H @ (D[:, None] * A_block.reshape(nb, -1)) / np.sqrt(d)


def sparse_rtt_positions(n, d, xi, seed):
    """SparseCol positions of the SparseRTT (Def. SparseCol): output row q < d takes xi distinct
    coordinates of [0, n), uniform without replacement (Floyd's algorithm on Philox stream 5, entity
    q), with Rademacher signs (bit t of the draw after the xi picks).  Returns (positions d x xi,
    signs d x xi in {+1, -1}), positions in insertion order."""
    return _ss.columns(d, n, xi, seed, stream=STREAM_SPARSECOL)


def sparse_rtt_apply(A, d, xi, seed):
    """Y = Omega^T A for the SparseRTT Omega = D F S (Def. SparseRTT) with F = H_n / sqrt(n):
    Y[q, :] = (d xi)^{-1/2} sum_t rho_qt (H_n D A)[s_qt, :] in float64."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    D = diag_signs(n, seed).astype(np.float64)
    HDA = fwht(D[:, None] * A.reshape(n, -1))
    pos, sg = sparse_rtt_positions(n, d, xi, seed)
    Y = np.zeros((d, HDA.shape[1]))
    for t in range(xi):
        Y += sg[:, t, None] * HDA[pos[:, t]]
    return Y / np.sqrt(d * xi)
