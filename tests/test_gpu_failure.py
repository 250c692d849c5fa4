"""Failure detection without a GPU fault: an injected allocation failure and a bounded wait that
runs out.

Neither test faults, traps or hangs the GPU.  The allocation failure is injected on the host
(RSK_FAULT_NOMEM=1 makes the workspace allocation report failure before calling the allocator).
The timeout shortens the iteration limit of the least-squares QR's reflector-ready polls (a
global-memory flag that the CTA owning the previous column publishes) to two polls, so the waiting
CTAs give up, record the timeout in the handle's device status word and return; the solver reports
RSK_ERR_TIMEOUT, and the same handle then solves correctly once the default limit is restored.
"""
import ctypes
import os

import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

RSK_ERR_NOMEM, RSK_ERR_TIMEOUT = 2, 5


@pytest.fixture
def fresh_handle():
    from paper_2508_21189_gb300 import _lib
    lib = _lib.load()
    torch.cuda.init()
    h = ctypes.c_void_p()
    assert lib.rsk_create(ctypes.byref(h)) == 0
    yield lib, h
    assert lib.rsk_destroy(h) == 0


def test_injected_workspace_failure_returns_nomem(fresh_handle, monkeypatch):
    lib, h = fresh_handle
    n, k, d = 4096, 64, 256
    A = torch.randn(n, k, device="cuda")
    SA = torch.empty(d, k, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    monkeypatch.setenv("RSK_FAULT_NOMEM", "1")
    st = lib.rsk_sparse_sign_apply(h, A.data_ptr(), 1, n, k, k, d, 8, 0, SA.data_ptr(), 1, k, stream)
    assert st == RSK_ERR_NOMEM
    assert b"RSK_FAULT_NOMEM" in lib.rsk_last_error(h)
    monkeypatch.delenv("RSK_FAULT_NOMEM")
    # nothing was launched and the handle is still usable
    assert lib.rsk_sparse_sign_apply(h, A.data_ptr(), 1, n, k, k, d, 8, 0, SA.data_ptr(), 1, k, stream) == 0
    assert lib.rsk_sync_status(h, stream) == 0
    assert torch.isfinite(SA).all()


def test_reflector_flag_wait_times_out(fresh_handle):
    import paper_2508_21189_gb300 as rsk
    lib, h = fresh_handle
    A, b = synthetic.batched_problem(20000, 64, seed=11, device="cuda", dtype=torch.float32)
    x = torch.empty(64, dtype=torch.float64, device="cuda")
    opts = rsk.LsqOpts(256, 8, 0, rsk.RSK_F32, rsk.RSK_F32, 1e-10, 4, 50, 1e-6, rsk.RSK_F64)
    info = rsk.LsqInfo()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def solve():
        return lib.rsk_lstsq_sketch_precond(h, A.data_ptr(), rsk.RSK_F32, A.shape[0], 64, 64, b.data_ptr(),
                                            x.data_ptr(), ctypes.byref(opts), ctypes.byref(info), stream)

    assert lib.rsk_set_wait_limit(h, 1) == 0
    assert solve() == RSK_ERR_TIMEOUT
    assert b"wait ran out" in lib.rsk_last_error(h)
    # the status word was read and cleared, the context is intact: the default limit solves
    assert lib.rsk_set_wait_limit(h, 0) == 0
    assert solve() == 0
    assert info.backward_err <= 1e-10
