"""GPU parity of the SparseRTT sketch (Def. SparseRTT, Def. SparseCol) against the oracle.

The SparseCol positions and signs must match bit for bit.  Y is compared column by column with
    ||(Y_gpu - Y_oracle)[:, c]||_2 <= 4 (u_in + (ceil(log2 n) + xi) u_32) sqrt(n/d) ||A[:, c]||_2,
the SRTT's bound with the xi-term sum of every output row added to the transform depth (u_in = 0
when the oracle sees the stored values).
"""
import math

import numpy as np
import pytest
import torch

from oracle import srtt as osr
import synthetic

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


def test_default_xi(rsk):
    assert rsk.rsk_sparse_rtt_default_xi(2048) == math.ceil(1.5 * math.log(2048))
    assert rsk.rsk_sparse_rtt_default_xi(1) == 1


@pytest.mark.parametrize("n,d,xi,seed", [(1, 1, 1, 0), (1024, 100, 4, 1), (1 << 16, 2048, 12, 2), (64, 2048, 32, 3)])
def test_draw_bit_exact(rsk, n, d, xi, seed):
    pos, bits = rsk.rsk_sparse_rtt_draw(n, d, seed, xi=xi)
    p, s = osr.sparse_rtt_positions(n, d, xi, seed)
    assert np.array_equal(pos.cpu().numpy(), p)
    got = bits.cpu().numpy().view(np.uint32)
    t = np.arange(xi, dtype=np.uint32)
    assert np.array_equal(np.where((got[:, None] >> t[None, :]) & 1, -1, 1), s)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,k,d,xi", [(1, 1, 1, 1), (2048, 8, 64, 3), (4096, 13, 300, 0), (1 << 15, 40, 1000, 0),
                                      (1 << 16, 256, 2048, 0)])
def test_apply_parity(rsk, dtype, n, k, d, xi):
    A = synthetic.colscaled_gaussian(n, k, seed=n + k + 1, device="cuda", dtype=torch.float32).to(dtype)
    Y = rsk.rsk_sparse_rtt_apply(A, d, 9, xi=xi, out_dtype=torch.float64).cpu().numpy()
    xi = xi or rsk.rsk_sparse_rtt_default_xi(d)
    A64 = A.double().cpu().numpy()
    ref = osr.sparse_rtt_apply(A64, d, xi, 9)
    L = max(1, math.ceil(math.log2(max(n, 2))))
    bound = 4 * (L + xi) * U32 * math.sqrt(n / d) * np.linalg.norm(A64, axis=0)
    err = np.linalg.norm(Y - ref, axis=0)
    assert np.all(err <= bound + 1e-300), float((err / np.maximum(bound, 1e-300)).max())


def test_rejects_bad_sizes(rsk):
    A = torch.randn(1000, 4, device="cuda")
    with pytest.raises(Exception):
        rsk.rsk_sparse_rtt_apply(A, 64, 1)          # n not a power of two
    A = torch.randn(1024, 4, device="cuda")
    with pytest.raises(Exception):
        rsk.rsk_sparse_rtt_apply(A, 4096, 1)        # more output rows than the gather holds
    with pytest.raises(Exception):
        rsk.rsk_sparse_rtt_apply(A, 64, 1, xi=33)   # xi above 32
