"""GPU parity of the sparse sign embedding (generation, inverted index, S @ A) against the oracle.

Integers (rows, signs, the inverted index) must match bit for bit.  Floating point:
  * F64 input: |SA_gpu - SA_oracle| <= 1e-12 * (|S| |A|) elementwise.
  * F32 / BF16 input, oracle on the unrounded values:
        ||(SA_gpu - SA_oracle)[i, :]||_2 <= 4 u sqrt(zeta) ||(|S| |A|)[i, :]||_2,
    u the storage unit roundoff (2^-24 for F32, 2^-8 for BF16).
  * BF16 input, oracle on the rounded values (only FP32 accumulation differs): the same row
    bound with u = 2^-24, which any index or sign error would break.
"""
import numpy as np
import pytest
import torch

from oracle import sparse_sign as osk
import synthetic

pytestmark = pytest.mark.gpu

U = {torch.float32: 2.0 ** -24, torch.bfloat16: 2.0 ** -8}


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    assert torch.cuda.is_available()
    return m


def global_csr_from_chunks(offs, ents, n, d, zeta, chunk):
    """Concatenate the chunked index (chunks in order) into one CSR (rowptr, cols, neg)."""
    offs = offs.cpu().numpy().view(np.uint16).astype(np.int64)
    ents = ents.cpu().numpy().view(np.uint16).astype(np.int64)
    nch = offs.shape[0]
    rows_l, chunk_l, pos_l, j_l, neg_l = [], [], [], [], []
    for c in range(nch):
        o = offs[c, : d + 1]
        assert np.all(offs[c, d:] == o[-1])
        cnt = np.diff(o)
        assert o[0] == 0 and np.all(cnt >= 0)
        m = int(o[-1])
        blk = ents[c * chunk * zeta: c * chunk * zeta + m]
        rows_l.append(np.repeat(np.arange(d), cnt))
        chunk_l.append(np.full(m, c))
        pos_l.append(np.arange(m))
        j_l.append(c * chunk + (blk & 0x7FFF))
        neg_l.append(blk >> 15)
    r = np.concatenate(rows_l)
    order = np.lexsort((np.concatenate(pos_l), np.concatenate(chunk_l), r))
    j = np.concatenate(j_l)[order]
    neg = np.concatenate(neg_l)[order].astype(bool)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=d), out=rowptr[1:])
    return rowptr, j, neg


@pytest.mark.parametrize("n,d,zeta,seed", [(20000, 400, 8, 0), (1, 1, 1, 3), (769, 7, 7, 5), (3001, 40, 32, 7),
                                           (5000, 8192, 8, 9), (2000, 64, 13, 11), (1537, 2048, 8, 2**40 + 5)])
def test_generate_and_index_bit_exact(rsk, n, d, zeta, seed):
    rows, bits = rsk.rsk_sparse_sign_generate(n, d, zeta, seed)
    o_rows, o_signs = osk.columns(n, d, zeta, seed)
    assert np.array_equal(rows.cpu().numpy(), o_rows)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), osk.sign_bits(o_signs))
    chunk, nch, pitch = rsk.rsk_sparse_sign_index_dims(n, d, zeta)
    assert pitch >= d + 1 and pitch % 8 == 0
    offs, ents = rsk.rsk_sparse_sign_index(n, d, zeta, seed)
    rowptr, j, neg = global_csr_from_chunks(offs, ents, n, d, zeta, chunk)
    o_rowptr, o_j, o_neg = osk.csr(n, d, zeta, seed)
    assert np.array_equal(rowptr, o_rowptr)
    assert np.array_equal(j, o_j)
    assert np.array_equal(neg, o_neg)


def check_f64(SA, A64, d, zeta, seed):
    ref = osk.apply(A64, d, zeta, seed)
    scale = osk.abs_apply(A64, d, zeta, seed) / np.sqrt(zeta)
    err = np.abs(SA - ref)
    assert np.all(err <= 1e-12 * scale + 1e-300), float((err / np.maximum(scale, 1e-300)).max())


def check_rows(SA, A_ref, d, zeta, seed, u):
    ref = osk.apply(A_ref, d, zeta, seed)
    scale = osk.abs_apply(A_ref, d, zeta, seed) / np.sqrt(zeta)
    num = np.linalg.norm(SA - ref, axis=1)
    bound = 4 * u * np.sqrt(zeta) * np.linalg.norm(scale, axis=1)
    assert np.all(num <= bound + 1e-300), float((num / np.maximum(bound, 1e-300)).max())


def test_f64_small_config(rsk):
    # A 20000 x 100 N(0,1) float64, d = 400, zeta = 8 (the plain FP64 configuration)
    A = synthetic.gaussian(20000, 100, seed=8, device="cuda", dtype=torch.float64)
    SA = rsk.rsk_sparse_sign_apply(A, 400, 8, 0, out_dtype=torch.float64)
    check_f64(SA.cpu().numpy(), A.cpu().numpy(), 400, 8, 0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,k,d,zeta", [(5000, 256, 2048, 8), (1537, 33, 77, 4), (769, 65, 7, 7), (3, 1, 2, 1),
                                         (12000, 100, 2000, 8)])
def test_lowp_parity(rsk, dtype, n, k, d, zeta):
    A32 = synthetic.colscaled_gaussian(n, k, seed=n + k, device="cuda", dtype=torch.float32)
    A = A32.to(dtype)
    SA = rsk.rsk_sparse_sign_apply(A, d, zeta, 123).cpu().numpy().astype(np.float64)
    check_rows(SA, A32.double().cpu().numpy(), d, zeta, 123, U[dtype])        # vs unrounded
    check_rows(SA, A.double().cpu().numpy(), d, zeta, 123, 2.0 ** -24)       # vs rounded input


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_strided_and_unaligned(rsk, dtype):
    n, k, d, zeta = 3000, 37, 50, 8
    base = synthetic.gaussian(n, k + 5, seed=4, device="cuda", dtype=torch.float64).to(dtype)
    views = [base[:, :k],                      # lda = k + 5 (TMA only if lda*esize % 16 == 0)
             base[:, 1:k + 1]]                 # base pointer offset by one element -> fallback path
    for A in views:
        SA = rsk.rsk_sparse_sign_apply(A, d, zeta, 77, out_dtype=torch.float64)
        A64 = A.double().cpu().numpy()
        if dtype == torch.float64:
            check_f64(SA.cpu().numpy(), A64, d, zeta, 77)
        else:
            check_rows(SA.cpu().numpy(), A64, d, zeta, 77, 2.0 ** -24)


def test_output_leading_dimension_and_plan(rsk):
    n, k, d, zeta = 4000, 40, 300, 8
    A = synthetic.gaussian(n, k, seed=5, device="cuda", dtype=torch.float32)
    big = torch.full((d, k + 7), 7.0, device="cuda", dtype=torch.float32)
    out = big[:, :k]
    rsk.rsk_sparse_sign_apply(A, d, zeta, 9, out=out)
    assert torch.all(big[:, k:] == 7.0)
    plan = rsk.rsk_sparse_sign_plan_create(n, d, zeta, 9)
    via_plan = plan.apply(A)
    plan.close()
    assert torch.equal(via_plan, out)


def test_deterministic(rsk):
    A = synthetic.colscaled_gaussian(50000, 256, seed=1, device="cuda", dtype=torch.bfloat16)
    a = rsk.rsk_sparse_sign_apply(A, 2048, 8, 42)
    b = rsk.rsk_sparse_sign_apply(A, 2048, 8, 42)
    assert torch.equal(a, b)


def test_invalid_arguments(rsk):
    A = torch.zeros(10, 4, device="cuda")
    with pytest.raises(rsk.RskError) as e:
        rsk.rsk_sparse_sign_apply(A, 4, 8, 0)          # zeta > d
    assert e.value.status == 1
    with pytest.raises(rsk.RskError):
        rsk.rsk_sparse_sign_apply(A, 9000, 8, 0)       # d beyond the supported range
    rsk.rsk_sync_status()


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_full_size_embedding(rsk, dtype):
    """A 2^22 x 256 (entries N(0,1) x logspaced column scales), d = 2048, zeta = 8, in the
    launch configuration the benchmark times: integer index bit-exact, sampled columns of SA
    against the oracle."""
    n, k, d, zeta, seed = 1 << 22, 256, 2048, 8, 0
    A32 = synthetic.colscaled_gaussian(n, k, seed=2022, device="cuda", dtype=torch.float32)
    A = A32.to(dtype)
    SA = rsk.rsk_sparse_sign_apply(A, d, zeta, seed).cpu().numpy().astype(np.float64)
    cols = [0, 1, 63, 64, 127, 200, 255]
    sub32 = A32[:, cols].double().cpu().numpy()
    subr = A[:, cols].double().cpu().numpy()
    check_rows(SA[:, cols], sub32, d, zeta, seed, U[dtype])
    check_rows(SA[:, cols], subr, d, zeta, seed, 2.0 ** -24)
    if dtype == torch.bfloat16:
        chunk, _, _ = rsk.rsk_sparse_sign_index_dims(n, d, zeta)
        offs, ents = rsk.rsk_sparse_sign_index(n, d, zeta, seed)
        rowptr, j, neg = global_csr_from_chunks(offs, ents, n, d, zeta, chunk)
        o_rowptr, o_j, o_neg = osk.csr(n, d, zeta, seed)
        assert np.array_equal(rowptr, o_rowptr)
        assert np.array_equal(j, o_j) and np.array_equal(neg, o_neg)


def _split_reference(a):
    """hi = RN32(a), lo = RN32(a - hi), with the library's flush rules outside the FP32 normal range."""
    tiny = np.float64(2.0 ** -126)
    with np.errstate(over="ignore", invalid="ignore"):
        hi = a.astype(np.float32)
        lo = (a - hi.astype(np.float64)).astype(np.float32)
    small = np.abs(a) < tiny
    hi = np.where(small, np.copysign(np.float32(0), a).astype(np.float32), hi)
    lo = np.where(small | (np.abs(lo.astype(np.float64)) < tiny) | ~np.isfinite(hi), np.float32(0), lo)
    return hi, lo


def test_split_pairs_bit_exact(rsk):
    rng = np.random.default_rng(11)
    a = rng.standard_normal(200000) * np.exp2(rng.integers(-130, 130, 200000).astype(np.float64))
    # exact ties: an FP32 value plus half of its ulp (round to even either way), and near-ties
    base = rng.standard_normal(4000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(base).astype(np.float32)).astype(np.float64)
    extra = np.concatenate([base + ulp / 2, base - ulp / 2, base + ulp / 2 * (1 + 2.0 ** -25), base + ulp / 2 * (1 - 2.0 ** -25),
                            [0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.5e38, -1e300, 1e-310, 2.0 ** -126,
                             2.0 ** -127, 1.0 + 2.0 ** -40, np.finfo(np.float32).max * (1 + 2.0 ** -25)]])
    a = np.concatenate([a, extra])
    A = torch.from_numpy(a.reshape(-1, 1)).cuda()
    P = rsk.rsk_split_pairs(A).cpu().numpy().reshape(-1, 2)
    hi, lo = _split_reference(a)
    assert np.array_equal(P[:, 0].view(np.uint32), hi.view(np.uint32))
    assert np.array_equal(P[:, 1].view(np.uint32), lo.view(np.uint32))
    # the pair carries a to 2^-48 relative wherever lo cannot be flushed (|a - hi| < 2^-126 only when
    # that is below 2^-56 |a|)
    ok = (np.abs(a) > 2.0 ** -70) & (np.abs(a) < 2.0 ** 126)
    err = np.abs(P[ok, 0].astype(np.float64) + P[ok, 1].astype(np.float64) - a[ok])
    assert np.all(err <= 2.0 ** -48 * np.abs(a[ok]))


def test_pairs_apply_parity(rsk):
    # double-float accumulation of the split pairs against the FP64 oracle: the pair carries 2^-48
    # relative per entry and the sum ~2^-44 relative per accumulated row
    n, k, d, zeta = 30000, 50, 400, 8
    A = synthetic.gaussian(n, k, seed=12, device="cuda", dtype=torch.float64)
    P = rsk.rsk_split_pairs(A)
    SA = rsk.rsk_sparse_sign_apply_pairs(P, d, zeta, 5).cpu().numpy()
    check_rows(SA, A.cpu().numpy(), d, zeta, 5, 2.0 ** -40)


@pytest.mark.parametrize("dtype,n,k,d", [(torch.bfloat16, 1 << 20, 256, 2048), (torch.float32, 300001, 37, 100),
                                         (torch.float64, 5000, 12, 64)])
def test_host_input_apply(rsk, dtype, n, k, d):
    # A streamed from pinned host memory in row blocks (several blocks for the 2^20-row case, a ragged
    # last block, an odd k that takes the plain-load path): equal to the device-input apply up to the
    # regrouping of the partial sums, and against the oracle on sampled columns
    A32 = synthetic.colscaled_gaussian(n, k, seed=n + k, device="cpu", dtype=torch.float32)
    A = A32.to(dtype).pin_memory()
    out_dt = torch.float64 if dtype == torch.float64 else torch.float32
    SA_h = rsk.rsk_sparse_sign_apply_host(A, d, 8, 77, out_dtype=out_dt)
    SA_d = rsk.rsk_sparse_sign_apply(A.cuda(), d, 8, 77, out_dtype=out_dt)
    torch.cuda.synchronize()
    diff = (SA_h.double() - SA_d.double()).abs().max().item()
    scale = SA_d.double().abs().max().item()
    assert diff <= (1e-12 if dtype == torch.float64 else 1e-5) * scale, diff
    cols = list(range(min(k, 3)))
    check_rows(SA_h.double().cpu().numpy()[:, cols], A.double().numpy()[:, cols], d, 8, 77, 2.0 ** -24)
