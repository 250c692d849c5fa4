"""The tcgen05 BF16 GEMM against a plain FP64 product of the same BF16 values.

D = A B^T with FP32 accumulation: every element within 1e-5 (|A| |B|^T) + 1e-30 of the FP64 product
(FP32 accumulation over K terms, in tensor-core order).  Shapes span one tile, ragged M, K and N
(out-of-bounds rows and columns are zero-filled by the copies), the RSVD's N = 300, and split K.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


@pytest.mark.parametrize("M,K,N,nsplit", [(128, 64, 32, 1), (256, 128, 64, 1), (128, 64, 320, 1), (1000, 1000, 300, 1),
                                          (4096, 2048, 300, 1), (777, 4104, 45, 1), (1024, 16384, 320, 4),
                                          (8192, 8192, 300, 2), (300, 512, 512, 1)])
def test_gemm_matches_fp64(rsk, M, K, N, nsplit):
    g = torch.Generator(device="cuda")
    g.manual_seed(M + K + N)
    A = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    D = rsk.rsk_gemm_bf16(A, B, nsplit=nsplit)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    ref = A.double() @ B.double().T
    scale = A.double().abs() @ B.double().abs().T
    err = (D.double() - ref).abs()
    assert bool((err <= 1e-5 * scale + 1e-30).all()), float((err / scale.clamp_min(1e-30)).max())
