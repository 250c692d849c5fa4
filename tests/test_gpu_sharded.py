"""GPU parity of the row-sharded sketch on one GPU: the ranks' row blocks are sketched one after
another through the C ABI (rsk_sparse_sign_apply_rows / rsk_srtt_apply_rows), summed in rank order
by rsk_sketch_sum_partials, and compared with the oracle -- each partial with the oracle's
row-block form, the sum with the oracle's whole-matrix sketch.  (Ranks whose kernels wait on one
another never share a GPU; these partials are independent, so running them in turn is exact.)
"""
import math

import numpy as np
import pytest
import torch

from oracle import sparse_sign as osk
from oracle import srtt as osr
import synthetic

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("world", [2, 3])
def test_sparse_sign_row_shards(rsk, dtype, world):
    from paper_2508_21189_gb300.sharded import row_partition
    n, k, d, zeta, seed = 50_000, 96, 400, 8, 21
    A = synthetic.colscaled_gaussian(n, k, seed=5, device="cuda", dtype=torch.float32).to(dtype)
    A64 = A.double().cpu().numpy()
    out_dt = torch.float64 if dtype == torch.float64 else torch.float32
    parts = []
    for r0, nr in row_partition(n, world, 1):
        p = rsk.rsk_sparse_sign_apply_rows(A[r0:r0 + nr], r0, d, zeta, seed, out_dtype=out_dt)
        ref = osk.apply_block(A64[r0:r0 + nr], r0, d, zeta, seed)
        err = np.abs(p.double().cpu().numpy() - ref)
        scale = osk.abs_apply_block(A64[r0:r0 + nr], r0, d, zeta, seed) / math.sqrt(zeta)  # |S||A|
        if dtype == torch.float64:
            assert np.all(err <= 1e-12 * scale + 1e-300)
        else:
            bound = 4 * U32 * math.sqrt(zeta) * np.linalg.norm(scale, axis=1)
            assert np.all(np.linalg.norm(err, axis=1) <= bound + 1e-300)
        parts.append(p)
    total = rsk.rsk_sketch_sum_partials(torch.stack(parts))
    # the rank-ordered sum, element by element
    seq = parts[0].clone()
    for p in parts[1:]:
        seq += p
    assert torch.equal(total, seq)
    whole = osk.apply(A64, d, zeta, seed)
    scale = osk.abs_apply(A64, d, zeta, seed) / math.sqrt(zeta)
    err = np.abs(total.double().cpu().numpy() - whole)
    if dtype == torch.float64:
        assert np.all(err <= 1e-12 * scale + 1e-300)
    else:
        assert np.all(np.linalg.norm(err, axis=1) <= 4 * U32 * math.sqrt(zeta) * np.linalg.norm(scale, axis=1))


def test_rows_at_zero_is_the_whole_apply(rsk):
    A = synthetic.colscaled_gaussian(30_000, 64, seed=8, device="cuda", dtype=torch.bfloat16)
    a = rsk.rsk_sparse_sign_apply(A, 512, 8, 3)
    b = rsk.rsk_sparse_sign_apply_rows(A, 0, 512, 8, 3)
    assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_srtt_row_shards(rsk, dtype):
    from paper_2508_21189_gb300.sharded import row_partition
    n, k, d, seed = 1 << 15, 24, 700, 6
    A = synthetic.colscaled_gaussian(n, k, seed=9, device="cuda", dtype=torch.float32).to(dtype)
    A64 = A.double().cpu().numpy()
    parts = []
    for r0, nr in row_partition(n, 3, 2048):
        parts.append(rsk.rsk_srtt_apply_rows(A[r0:r0 + nr], r0, n, d, seed))
        ref = osr.apply_block(A64[r0:r0 + nr], r0, n, d, seed)
        got = parts[-1].double().cpu().numpy()
        bound = 4 * 15 * U32 * math.sqrt(n / d) * np.linalg.norm(A64[r0:r0 + nr], axis=0)
        assert np.all(np.linalg.norm(got - ref, axis=0) <= bound)
    total = rsk.rsk_sketch_sum_partials(torch.stack(parts)).double().cpu().numpy()
    whole = osr.apply(A64, d, seed)
    bound = 4 * (15 + 3) * U32 * math.sqrt(n / d) * np.linalg.norm(A64, axis=0)
    assert np.all(np.linalg.norm(total - whole, axis=0) <= bound)


def test_srtt_rows_rejects_unaligned_block(rsk):
    A = torch.randn(4096, 8, device="cuda")
    with pytest.raises(Exception):
        rsk.rsk_srtt_apply_rows(A[:2048], 1000, 4096, 64, 1)
    with pytest.raises(Exception):
        rsk.rsk_srtt_apply_rows(A, 2048, 4096, 64, 1)  # block runs past n
