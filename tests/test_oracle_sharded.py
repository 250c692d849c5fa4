"""The row-sharded sketch on CPU: the oracle's row-block forms against the whole
sketch, and the sharding driver's gather + rank-ordered sum over two gloo ranks.

Pins: a sketch is linear in A, so for any row partition the block contributions must sum to the
oracle's whole-matrix sketch (exactly so up to FP64 rounding); the sparse sign's first block with
col0 = 0 is the whole-matrix sketch of that block.  The distributed reduction must return, on every
rank, bit for bit the rank-ordered sum of the same partials computed in one process.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import sparse_sign as osk
from oracle import srtt as osr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ordered_sum(parts):
    out = parts[0].clone()
    for g in range(1, parts.shape[0]):
        out += parts[g]
    return out


@pytest.mark.parametrize("world,align", [(2, 1), (3, 1), (4, 768), (5, 7)])
def test_partition_covers_rows(world, align):
    from paper_2508_21189_gb300.sharded import row_partition
    n = 10_000
    blocks = row_partition(n, world, align)
    assert len(blocks) == world
    assert blocks[0][0] == 0 and sum(r for _, r in blocks) == n
    for (r0, nr), (r1, _) in zip(blocks, blocks[1:]):
        assert r0 + nr == r1 and r0 % align == 0
    assert max(r for _, r in blocks) - min(r for _, r in blocks) <= align


def test_sparse_sign_blocks_sum_to_whole():
    rng = np.random.default_rng(3)
    n, k, d, zeta, seed = 3000, 7, 64, 8, 11
    A = rng.standard_normal((n, k))
    whole = osk.apply(A, d, zeta, seed)
    cuts = [0, 1, 700, 701, 2048, n]
    parts = [osk.apply_block(A[a:b], a, d, zeta, seed) for a, b in zip(cuts, cuts[1:])]
    scale = osk.abs_apply(A, d, zeta, seed) / np.sqrt(zeta)
    assert np.all(np.abs(sum(parts) - whole) <= 1e-13 * scale + 1e-300)
    # the absolute-value form sums the same way, and is the whole abs_apply at col0 = 0
    abs_parts = [osk.abs_apply_block(A[a:b], a, d, zeta, seed) for a, b in zip(cuts, cuts[1:])]
    np.testing.assert_allclose(sum(abs_parts), osk.abs_apply(A, d, zeta, seed), rtol=1e-13, atol=0)
    assert np.all(sum(abs_parts) >= np.abs(whole) * np.sqrt(zeta) * (1 - 1e-13))
    # col0 = 0 is the whole-matrix sketch of that block; a block elsewhere uses other columns of S
    np.testing.assert_allclose(osk.apply_block(A[:700], 0, d, zeta, seed), osk.apply(A[:700], d, zeta, seed),
                               rtol=0, atol=1e-14)
    assert not np.allclose(osk.apply_block(A[:700], 700, d, zeta, seed), osk.apply(A[:700], d, zeta, seed))


def test_srtt_blocks_sum_to_whole():
    rng = np.random.default_rng(4)
    n, k, d, seed = 8192, 5, 100, 2
    A = rng.standard_normal((n, k))
    whole = osr.apply(A, d, seed)
    parts = [osr.apply_block(A[a:a + 2048], a, n, d, seed) for a in range(0, n, 2048)]
    np.testing.assert_allclose(sum(parts), whole, rtol=0, atol=1e-12 * np.abs(A).sum(0).max())
    # a single block covering everything is the definition itself
    np.testing.assert_allclose(osr.apply_block(A, 0, n, d, seed), whole, rtol=0, atol=1e-12 * np.abs(A).sum(0).max())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle import sparse_sign as osk_
    from oracle import srtt as osr_
    from paper_2508_21189_gb300.sharded import reduce_partials, row_partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(9)
    n, k, d = 8192, 6, 96
    A = rng.standard_normal((n, k))  # every rank draws the same A and keeps its own rows
    align = 2048 if kind == "srtt" else 1
    r0, nr = row_partition(n, world, align)[rank]
    if kind == "srtt":
        part = osr_.apply_block(A[r0:r0 + nr], r0, n, d, 5)
    else:
        part = osk_.apply_block(A[r0:r0 + nr], r0, d, 8, 5)
    got = reduce_partials(torch.from_numpy(part), _ordered_sum)
    out[rank] = got.numpy()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["sparse_sign", "srtt"])
def test_two_rank_gloo_reduction_is_rank_ordered_sum(kind):
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), kind, out), nprocs=world, start_method="spawn",
                       join=True)
    rng = np.random.default_rng(9)
    n, k, d = 8192, 6, 96
    A = rng.standard_normal((n, k))
    from paper_2508_21189_gb300.sharded import row_partition
    blocks = row_partition(n, world, 2048 if kind == "srtt" else 1)
    if kind == "srtt":
        parts = [osr.apply_block(A[a:a + m], a, n, d, 5) for a, m in blocks]
        whole = osr.apply(A, d, 5)
    else:
        parts = [osk.apply_block(A[a:a + m], a, d, 8, 5) for a, m in blocks]
        whole = osk.apply(A, d, 8, 5)
    ref = _ordered_sum(torch.from_numpy(np.stack(parts))).numpy()
    for r in range(world):
        assert np.array_equal(out[r], ref), "distributed sum differs from the rank-ordered sum"
    np.testing.assert_allclose(ref, whole, rtol=0, atol=1e-12 * np.abs(A).sum(0).max())
