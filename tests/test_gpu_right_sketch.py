"""GPU parity of the right sketch Y = A Omega = A S^T (rsk_sparse_sign_apply_right) with the FP64
oracle's S: SparseUniform on its own Philox stream and on the RSVD's stream 3, and SparseStack.

Y[i, c] = zeta^{-1/2} sum over the entries (j, sign) of row c of S of sign * A[i, j], accumulated in
FP32: every element within 1e-5 (|A| |S|^T) zeta^{-1/2} + 1e-30 of the FP64 product with the same S.
Sizes span several 32-row tiles and index chunks with ragged tails.
"""
import numpy as np
import pytest
import torch

from oracle import sparse_sign as osk
from oracle import sparse_stack as ost

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


@pytest.mark.parametrize("n,dc,k,zeta,kind,stream", [(1000, 3000, 64, 8, 0, -1), (777, 5000, 300, 8, 0, 3),
                                                     (2048, 1537, 200, 4, 1, -1), (33, 769, 17, 1, 0, -1),
                                                     (300, 20000, 512, 8, 0, -1)])
def test_right_sketch_matches_oracle(rsk, n, dc, k, zeta, kind, stream):
    g = torch.Generator().manual_seed(n + dc + k)
    A = torch.randn(n, dc, generator=g) * torch.logspace(-2, 0, dc)[None, :]
    Y = rsk.rsk_sparse_sign_apply_right(A.cuda(), k, zeta, seed=11, kind=kind, philox_stream=stream)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    if kind == 1:
        S = ost.matrix(dc, k, zeta, 11)
    else:
        S = osk.matrix(dc, k, zeta, 11, stream=osk.STREAM_LEFT if stream < 0 else stream)
    A64 = A.double().numpy()
    ref = np.asarray(S @ A64.T).T / np.sqrt(zeta)
    scale = np.asarray(abs(S) @ np.abs(A64).T).T / np.sqrt(zeta)
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert Y.shape == (n, k)
    assert np.all(err <= 1e-5 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())


def test_right_sketch_rsvd_omega(rsk):
    """Stream 3 is the RSVD's test matrix: Y = A Omega with the oracle's Omega."""
    from oracle import rsvd as orsvd
    g = torch.Generator().manual_seed(5)
    A = torch.randn(500, 4000, generator=g)
    Y = rsk.rsk_sparse_sign_apply_right(A.cuda(), 75, 8, seed=5, philox_stream=3)
    torch.cuda.synchronize()
    ref = A.double().numpy() @ orsvd.omega(4000, 75, 8, 5)
    assert np.abs(Y.double().cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()


def test_right_sketch_invalid(rsk):
    A = torch.zeros(64, 1000, device="cuda")
    with pytest.raises(rsk.RskError):
        rsk.rsk_sparse_sign_apply_right(A, 513, 8, seed=0)          # k beyond 512
    with pytest.raises(rsk.RskError):
        rsk.rsk_sparse_sign_apply_right(A, 64, 8, seed=0, kind=2)   # no such kind
    with pytest.raises(rsk.RskError):
        rsk.rsk_sparse_sign_apply_right(A, 60, 8, seed=0, kind=1)   # SparseStack needs k % zeta == 0
    with pytest.raises(TypeError):
        rsk.rsk_sparse_sign_apply_right(A.double(), 64, 8, seed=0)  # FP32 A only
