"""The tcgen05 BF16 GEMM against a plain FP64 product of the same BF16 values.

D = A B^T with FP32 accumulation: every element within 1e-5 (|A| |B|^T) + 1e-30 of the FP64 product
(FP32 accumulation over K terms, in tensor-core order).  Shapes span one tile, ragged M, K and N
(out-of-bounds rows and columns are zero-filled by the copies), the RSVD's N = 300, and split K.
N runs as two MMA halves, the second up to 16 columns narrower than the first (N = 300: 160 + 144, N =
304 exactly, N = 305: 160 + 160; N = 45: 32 + 16), alone, in pairs and in fours of row tiles.
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
                                          (8192, 8192, 300, 2), (300, 512, 512, 1), (1000, 640, 200, 1),
                                          (513, 256, 450, 1), (640, 128, 161, 2), (1024, 1024, 304, 1),
                                          (1024, 1024, 305, 1), (100, 640, 45, 3)])
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


@pytest.mark.parametrize("M,K,N,nsplit,row_major", [(128, 64, 32, 1, False), (256, 192, 96, 1, True),
                                                    (1000, 1000, 300, 1, False), (8192, 20000, 300, 3, False),
                                                    (333, 4104, 45, 1, True), (8192, 8192, 320, 2, True),
                                                    (8192, 32768, 300, 7, False)])
def test_gemm_mn_major_a(rsk, M, K, N, nsplit, row_major):
    """op(A) = A^T read in place (A given K x M row-major), column- or row-major D."""
    g = torch.Generator(device="cuda")
    g.manual_seed(7 * M + K + N)
    At = torch.randn(K, M + (8 - M % 8) % 8, generator=g, device="cuda").to(torch.bfloat16)[:, :M]
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    D = rsk.rsk_gemm_bf16_ex(At, B, a_mn=True, row_major_out=row_major, nsplit=nsplit)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    ref = At.double().T @ B.double().T
    scale = At.double().abs().T @ B.double().abs().T
    err = (D.double() - ref).abs()
    assert bool((err <= 1e-5 * scale + 1e-30).all()), float((err / scale.clamp_min(1e-30)).max())


@pytest.mark.parametrize("a_mn,M,K,N,row_major", [(False, 63488, 2048, 300, False), (False, 63488, 2048, 300, True),
                                                  (True, 8192, 16384, 300, False), (False, 40000, 640, 161, False)])
def test_gemm_automatic_splits(rsk, a_mn, M, K, N, row_major):
    """nsplit 0: 63488 rows are 248 pairs of row tiles; with up to 76 pairs resident (152 SMs) the
    rounds leave a last one of at most 40 pairs, which runs split over K (its rows summed from
    partials); the 8192-row MN-major product splits K.  Every element within the FP32-accumulation
    bound of the FP64 product; rows before the last 40 pairs are computed as without splits and are
    bit-identical to the nsplit = 1 result."""
    g = torch.Generator(device="cuda")
    g.manual_seed(M + K + N + int(a_mn))
    if a_mn:
        A = torch.randn(K, M, generator=g, device="cuda").to(torch.bfloat16)
        Aop = A.double().T
    else:
        A = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
        Aop = A.double()
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    D = rsk.rsk_gemm_bf16_ex(A, B, a_mn=a_mn, row_major_out=row_major, nsplit=0)
    D1 = rsk.rsk_gemm_bf16_ex(A, B, a_mn=a_mn, row_major_out=row_major, nsplit=1)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    ref = Aop @ B.double().T
    scale = Aop.abs() @ B.double().abs().T
    for X in (D, D1):
        err = (X.double() - ref).abs()
        assert bool((err <= 1e-5 * scale + 1e-30).all()), float((err / scale.clamp_min(1e-30)).max())
    if M == 63488:
        first = (248 - 40) * 256
        assert torch.equal(D[:first], D1[:first])


def test_gemm_row_major_out(rsk):
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    A = torch.randn(1000, 640, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(300, 640, generator=g, device="cuda").to(torch.bfloat16)
    D = rsk.rsk_gemm_bf16_ex(A, B, row_major_out=True)
    Dc = rsk.rsk_gemm_bf16(A, B)
    torch.cuda.synchronize()
    assert D.is_contiguous() and torch.equal(D, Dc)        # the same accumulation, stored transposed


@pytest.mark.parametrize("a_mn,M,K,N,nsplit", [(False, 300, 262144, 300, 48), (False, 300, 20000, 300, 8),
                                               (True, 20000, 300, 300, 1), (True, 8192, 300, 256, 1),
                                               (False, 1000, 300, 77, 1), (True, 4100, 1000, 300, 2),
                                               (True, 1001, 301, 45, 1), (False, 333, 1001, 7, 2)])
def test_gemm_f32_accuracy(rsk, a_mn, M, K, N, nsplit):
    """Three-term BF16 splits: within FP32 rounding of the exact product of the FP32 inputs (the
    neglected split products are O(2^-24) relative; FP32 accumulation over K adds K u |A||B|)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(M + 3 * K + N)
    A = torch.randn(K, M, generator=g, device="cuda") if a_mn else torch.randn(M, K, generator=g, device="cuda")
    B = torch.randn(N, K, generator=g, device="cuda")
    D = rsk.rsk_gemm_f32(A, B, a_mn=a_mn, nsplit=nsplit)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    Aop = A.double().T if a_mn else A.double()
    ref = Aop @ B.double().T
    scale = Aop.abs() @ B.double().abs().T
    rel = ((D.double() - ref).abs() / scale).max().item()
    # FP32 accumulation: a few u_32 per term in the worst case; typically ~sqrt(K) u_32
    assert rel <= 64 * 2.0 ** -24 * max(1.0, K ** 0.5 / 8), rel
    # and far beyond what one BF16 product could give
    assert rel <= 1e-5


def test_gemm_f32_gram_symmetric_orthogonal(rsk):
    """X^T X of an orthonormal X (QR of a Gaussian, FP32) is I to FP32 accuracy."""
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    X, _ = torch.linalg.qr(torch.randn(50000, 300, generator=g, device="cuda", dtype=torch.float64))
    Xc = X.float().T.contiguous()          # column-major X = row-major X^T (300 x 50000)
    ref = X.float().double().T @ X.float().double()
    errs = {}
    for nsplit in (16, 160):
        G = rsk.rsk_gemm_f32(Xc, Xc, nsplit=nsplit)
        torch.cuda.synchronize()
        errs[nsplit] = (G.double() - ref).abs().max().item()
    # the accumulation truncates: the diagonal's bias follows the main term's K steps per split, up to
    # about 2^-24 each (nsplit 16: 196 steps, measured 7.7e-6; nsplit 160: 20 steps, 1.1e-6), plus the
    # round-to-nearest sum of the partials
    assert errs[16] <= 196 * 2.0 ** -24, errs
    assert errs[160] <= 2e-6, errs


@pytest.mark.parametrize("a_mn,M,K,N,nsplit", [(False, 1000, 1000, 300, 1), (True, 1000, 4096, 300, 2),
                                               (False, 4100, 640, 256, 1), (True, 8192, 8192, 300, 2),
                                               (False, 777, 4104, 512, 3)])
@pytest.mark.parametrize("cluster", [2, 4])
def test_gemm_cluster_multicast(rsk, a_mn, M, K, N, nsplit, cluster):
    """Row tiles in clusters of 2 or 4 share the B tile by multicast: the same accumulation as the
    unclustered product, so the results are identical; a row-tile count that is not a multiple of the
    cluster adds tiles beyond M that write nothing."""
    g = torch.Generator(device="cuda")
    g.manual_seed(M + K + N + cluster)
    A = torch.randn(K, M + (8 - M % 8) % 8, generator=g, device="cuda").to(torch.bfloat16)[:, :M] if a_mn else \
        torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    D1 = rsk.rsk_gemm_bf16_ex(A, B, a_mn=a_mn, nsplit=nsplit, cluster=1)
    Dc = rsk.rsk_gemm_bf16_ex(A, B, a_mn=a_mn, nsplit=nsplit, cluster=cluster)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    assert torch.equal(D1, Dc)
    Aop = A.double().T if a_mn else A.double()
    ref = Aop @ B.double().T
    scale = Aop.abs() @ B.double().abs().T
    assert bool(((Dc.double() - ref).abs() <= 1e-5 * scale + 1e-30).all())


def test_gemm_cluster_invalid(rsk):
    A = torch.zeros(256, 64, device="cuda", dtype=torch.bfloat16)
    B = torch.zeros(48, 64, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(rsk.RskError):
        rsk.rsk_gemm_bf16_ex(A, B, cluster=3)
    with pytest.raises(rsk.RskError):
        rsk.rsk_gemm_bf16_ex(A, B, cluster=4)       # N half 32: no cluster of 4 is built
