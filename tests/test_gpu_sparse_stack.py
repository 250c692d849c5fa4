"""GPU parity of the SparseStack sketch (Def. SparseStack) against the oracle.

The draw (rows and signs) must match bit for bit.  S @ A uses the sparse sign gather, so the
tolerances are those of the sparse sign apply:
  * F64 input: |SA_gpu - SA_oracle| <= 1e-12 * (|S| |A|) elementwise;
  * F32 / BF16 input, oracle on the stored (rounded) values: row-wise
        ||(SA_gpu - SA_oracle)[i, :]||_2 <= 4 u_32 sqrt(zeta) ||(|S| |A|)[i, :]||_2.
"""
import math

import numpy as np
import pytest
import torch

from oracle import sparse_stack as ost
import synthetic

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


@pytest.mark.parametrize("n,d,zeta,seed", [(1, 1, 1, 0), (5000, 400, 8, 1), (3001, 64, 32, 2), (2048, 2048, 8, 3),
                                           (777, 8190, 13, 2**33 + 1)])
def test_generate_bit_exact(rsk, n, d, zeta, seed):
    rows, bits = rsk.rsk_sparse_stack_generate(n, d, zeta, seed)
    r, s = ost.columns(n, d, zeta, seed)
    assert np.array_equal(rows.cpu().numpy(), r)
    got = bits.cpu().numpy().view(np.uint32)
    q = np.arange(zeta, dtype=np.uint32)
    assert np.array_equal(np.where((got[:, None] >> q[None, :]) & 1, -1, 1), s)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,k,d,zeta", [(1, 1, 8, 8), (20000, 100, 400, 8), (7001, 33, 96, 4), (60000, 256, 2048, 8)])
def test_apply_parity(rsk, dtype, n, k, d, zeta):
    A = synthetic.colscaled_gaussian(n, k, seed=n + k, device="cuda", dtype=torch.float32).to(dtype)
    out_dt = torch.float64 if dtype == torch.float64 else torch.float32
    SA = rsk.rsk_sparse_stack_apply(A, d, zeta, 5, out_dtype=out_dt).double().cpu().numpy()
    A64 = A.double().cpu().numpy()
    ref = ost.apply(A64, d, zeta, 5)
    scale = ost.abs_apply(A64, d, zeta, 5) / math.sqrt(zeta)
    err = np.abs(SA - ref)
    if dtype == torch.float64:
        assert np.all(err <= 1e-12 * scale + 1e-300)
    else:
        bound = 4 * U32 * math.sqrt(zeta) * np.linalg.norm(scale, axis=1)
        assert np.all(np.linalg.norm(err, axis=1) <= bound + 1e-300)


def test_rejects_d_not_multiple_of_zeta(rsk):
    A = torch.randn(100, 4, device="cuda")
    with pytest.raises(Exception):
        rsk.rsk_sparse_stack_apply(A, 30, 8, 0)
