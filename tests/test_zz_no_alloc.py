"""The allocation-free sparse sign apply (rsk_sparse_sign_apply_noalloc), called through the C ABI.

Some callers cannot allocate device memory at all (an application that owns every device buffer,
or code that must not allocate after start-up).  This entry point serves them from a fixed array in
device memory.  The test checks it against the ordinary entry point (which allocates its workspace
through a handle) on two calls in a row, so the second call reuses the array the first left
behind (bit-identical results, since the plan and the summation order are the same), checks that
invalid sizes are rejected before anything is sized or launched, and that a size needing more
scratch than the array holds is refused.  The file
name makes pytest collect it last.
"""
import ctypes

import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point():
    import paper_2508_21189_gb300 as rsk
    lib = rsk.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(20000, 100, 400, 8, 5, torch.float64, torch.float64),
             (60000, 256, 2048, 8, 6, torch.bfloat16, torch.float32)]
    for n, k, d, zeta, seed, dt, out_dt in cases:
        A = synthetic.colscaled_gaussian(n, k, seed=seed, device="cuda", dtype=torch.float32).to(dt)
        ref = rsk.rsk_sparse_sign_apply(A, d, zeta, seed, out_dtype=out_dt)
        for _ in range(2):
            out = torch.full((d, k), float("nan"), device="cuda", dtype=out_dt)
            st = lib.rsk_sparse_sign_apply_noalloc(A.data_ptr(), rsk._dt(A), n, k, A.stride(0), d, zeta, seed,
                                                   out.data_ptr(), rsk._dt(out), out.stride(0), stream)
            assert st == 0
            torch.cuda.synchronize()
            # same plan, grid and summation order as the allocating call: the same bits, also on
            # the second call, which starts from the array the first call left behind
            assert torch.equal(out, ref)


def test_noalloc_refuses_oversized_problem():
    import paper_2508_21189_gb300 as rsk
    lib = rsk.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, k, d = 1 << 22, 256, 2048        # index + partials need far more than the fixed array
    A = torch.empty(8, 8, device="cuda")  # never read: the size check comes first
    out = torch.empty(8, 8, device="cuda")
    st = lib.rsk_sparse_sign_apply_noalloc(A.data_ptr(), 1, n, k, k, d, 8, 0, out.data_ptr(), 1, k, stream)
    assert st == 6  # RSK_ERR_UNSUPPORTED
    # invalid sizes are rejected as invalid, not as too large (and never divide by zero while sizing)
    assert lib.rsk_sparse_sign_apply_noalloc(A.data_ptr(), 1, n, k, k, (1 << 32) - 3, 8, 0, out.data_ptr(), 1, k,
                                             stream) == 1
    assert lib.rsk_sparse_sign_apply_noalloc(A.data_ptr(), 1, n, k, k, 4, 8, 0, out.data_ptr(), 1, k, stream) == 1
