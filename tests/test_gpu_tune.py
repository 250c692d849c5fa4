"""The autotuner on the GPU: tuned launch parameters keep parity with the oracle.

A non-default value is forced into the table for each knob (row ranges of the gather apply, bands of
the SRTT, rows per tile of the batched solver) and the results are checked against the oracle with
the usual tolerances; the timing tuners run and record what they choose.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import lsq as olsq
from oracle import sparse_sign as osk
from oracle import srtt as osr
import synthetic

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture
def rsk():
    import paper_2508_21189_gb300 as m
    L = m.lib()
    L.rsk_tune_cache_clear()
    yield m
    L.rsk_tune_cache_clear()


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("ranges", [1, 7, 64])
def test_tuned_row_ranges_keep_parity(rsk, ranges):
    n, k, d, zeta = 200_000, 64, 1024, 8
    A = synthetic.colscaled_gaussian(n, k, seed=3, device="cuda", dtype=torch.bfloat16)
    assert rsk.lib().rsk_tune_cache_set(0, 2, n, k, d, sms(), ranges) == 0
    SA = rsk.rsk_sparse_sign_apply(A, d, zeta, 5).double().cpu().numpy()
    A64 = A.double().cpu().numpy()
    ref = osk.apply(A64, d, zeta, 5)
    scale = osk.abs_apply(A64, d, zeta, 5) / math.sqrt(zeta)
    bound = 4 * U32 * math.sqrt(zeta) * np.linalg.norm(scale, axis=1)
    assert np.all(np.linalg.norm(SA - ref, axis=1) <= bound)


@pytest.mark.parametrize("bands", [1, 3])
def test_tuned_srtt_bands_keep_parity(rsk, bands):
    n, k, d = 1 << 15, 24, 500
    A = synthetic.colscaled_gaussian(n, k, seed=4, device="cuda", dtype=torch.float32)
    assert rsk.lib().rsk_tune_cache_set(1, 1, n, k, d, sms(), bands) == 0
    Y = rsk.rsk_srtt_apply(A, d, 2, out_dtype=torch.float64).cpu().numpy()
    A64 = A.double().cpu().numpy()
    ref = osr.apply(A64, d, 2)
    bound = 4 * 15 * U32 * math.sqrt(n / d) * np.linalg.norm(A64, axis=0)
    assert np.all(np.linalg.norm(Y - ref, axis=0) <= bound)


def test_tuned_batch_tile_keeps_parity(rsk):
    ns, ks = [9000, 30000, 5000], [32, 64, 16]
    As, bs = [], []
    for i, (n, k) in enumerate(zip(ns, ks)):
        A, b = synthetic.batched_problem(n, k, seed=70 + i, device="cuda", dtype=torch.float32)
        As.append(A)
        bs.append(b)
    assert rsk.lib().rsk_tune_cache_set(2, 1, sum(ns), len(ns), 0, sms(), 1024) == 0
    xs, infos = rsk.rsk_lstsq_sketch_precond_batched(As, bs, sketch_dtype=torch.float32, inner_dtype=torch.float32)
    for A, b, x in zip(As, bs, xs):
        assert olsq.backward_error(A.double().cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()) <= 1e-10


def test_autotune_calls_record_their_choice(rsk):
    L = rsk.lib()
    h = rsk.handle()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    chosen, ms = ctypes.c_int32(-1), ctypes.c_double(0)
    n, k, d = 1 << 20, 256, 2048
    assert L.rsk_autotune_sketch(h, 0, 2, n, k, d, 8, ctypes.byref(chosen), ctypes.byref(ms), stream) == 0
    assert chosen.value >= 0 and ms.value > 0
    v = ctypes.c_int32(-1)
    L.rsk_tune_cache_get(0, 2, n, k, d, sms(), ctypes.byref(v))
    assert v.value == chosen.value
    assert L.rsk_autotune_sketch(h, 1, 2, n, k, d, 8, ctypes.byref(chosen), ctypes.byref(ms), stream) == 0
    assert chosen.value >= 0 and ms.value > 0
