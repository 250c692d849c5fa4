"""Injectivity and dilation of a sparse test matrix on the adversarial subspace Q = [e_1 ... e_r].

Paper: Fig. 2 (Sec. 1.5) and its discussion in Sec. 3: alpha = sigma_min^2(Omega^T Q) and
beta = sigma_max^2(Omega^T Q) with embedding dimension k (k = 2r in the figure).  Omega^T Q is the
first r columns of the k x d left sketch S, so alpha and beta are the extreme eigenvalues of
G = S_r^T S_r, computed here exactly (dense symmetric eigensolver) for sizes the CPU holds.

TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np

from . import sparse_sign as _ss
from . import sparse_stack as _st


def first_columns(r, k, zeta, seed, kind=1):
    """S_r (k x r, dense, entries 0 or +-zeta^{-1/2}): the first r columns of the sketch."""
    return _st.dense(r, k, zeta, seed) if kind == 1 else _ss.dense(r, k, zeta, seed)


def extremes(r, k, zeta, seed, kind=1):
    """(alpha, beta) = (lambda_min, lambda_max) of S_r^T S_r."""
    S = first_columns(r, k, zeta, seed, kind)
    ev = np.linalg.eigvalsh(S.T @ S)
    return float(ev[0]), float(ev[-1])
