"""GPU parity of the SRTT (row a4) against the oracle.

P and D must match bit for bit.  Y is compared column by column with the bound
    ||(Y_gpu - Y_oracle)[:, c]||_2 <= 4 (u_in + ceil(log2 n) u_32) sqrt(n/d) ||A[:, c]||_2,
u_in the storage unit roundoff (0 when the oracle sees the rounded input), the oracle taking the
same stored values in FP64.
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


def check_cols(Y, A64, d, seed, u_in):
    n = A64.shape[0]
    ref = osr.apply(A64, d, seed)
    num = np.linalg.norm(Y - ref, axis=0)
    bound = 4 * (u_in + max(1, math.ceil(math.log2(max(n, 2)))) * U32) * math.sqrt(n / d) * np.linalg.norm(A64, axis=0)
    assert np.all(num <= bound + 1e-300), float((num / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("n,d,seed", [(1, 1, 0), (2, 2, 1), (1024, 100, 2), (4096, 2048, 3), (1 << 16, 3000, 4),
                                      (1 << 20, 2048, 5)])
def test_draw_bit_exact(rsk, n, d, seed):
    rows, bits = rsk.rsk_srtt_draw(n, d, seed)
    assert np.array_equal(rows.cpu().numpy(), osr.subsample(n, d, seed))
    D = osr.diag_signs(n, seed)
    got = bits.cpu().numpy().view(np.uint32)
    i = np.arange(n)
    gbit = (got[i >> 5] >> (i & 31).astype(np.uint32)) & 1
    assert np.array_equal(np.where(gbit == 1, -1, 1), D)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,k,d", [(1, 1, 1), (8, 3, 8), (1024, 13, 100), (2048, 8, 2048), (4096, 17, 2048),
                                   (1 << 15, 40, 1000), (1 << 16, 256, 2048)])
def test_apply_parity(rsk, dtype, n, k, d):
    A32 = synthetic.colscaled_gaussian(n, k, seed=n + k, device="cuda", dtype=torch.float32)
    A = A32.to(dtype)
    Y = rsk.rsk_srtt_apply(A, d, 7, out_dtype=torch.float64).cpu().numpy()
    check_cols(Y, A.double().cpu().numpy(), d, 7, 0.0)
    u_in = 2.0 ** -8 if dtype == torch.bfloat16 else 0.0
    check_cols(Y, A32.double().cpu().numpy(), d, 7, u_in)


def test_orthogonal_when_not_subsampled(rsk):
    n, k = 2048, 16
    A = synthetic.gaussian(n, k, seed=3, device="cuda", dtype=torch.float32)
    Y = rsk.rsk_srtt_apply(A, n, 11, out_dtype=torch.float64).cpu().numpy()
    A64 = A.double().cpu().numpy()
    assert np.allclose(Y.T @ Y, A64.T @ A64, rtol=1e-5, atol=1e-3)


def test_invalid(rsk):
    A = torch.zeros(1000, 4, device="cuda")
    with pytest.raises(rsk.RskError):
        rsk.rsk_srtt_apply(A, 10, 0)                 # n not a power of two
    A = torch.zeros(1024, 4, device="cuda")
    with pytest.raises(rsk.RskError):
        rsk.rsk_srtt_apply(A, 2000, 0)               # d > n


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_full_size_sampled_rows(rsk, dtype):
    """A 2^22 x 256, d = 2048 in the benchmark's launch configuration: sampled output rows against
    the oracle's one-row-at-a-time definition."""
    n, k, d, seed = 1 << 22, 256, 2048, 0
    A32 = synthetic.colscaled_gaussian(n, k, seed=2022, device="cuda", dtype=torch.float32)
    A = A32.to(dtype)
    Y = rsk.rsk_srtt_apply(A, d, seed, out_dtype=torch.float64).cpu().numpy()
    rows = [0, 1, 777, 2047]
    cols = list(range(0, 256, 37))
    A64 = A[:, cols].double().cpu().numpy()
    ref = osr.apply_rows(A64, rows, d, seed)
    err = np.abs(Y[np.ix_(rows, cols)] - ref)
    bound = 4 * 22 * U32 * math.sqrt(n / d) * np.linalg.norm(A64, axis=0)[None, :]
    assert np.all(err <= bound), float((err / bound).max())
