"""GPU parity of the randomized SVD with a sparse sign test matrix (row a9).

Reduced twin (oracle-feasible): A = U diag(j^-2, j <= rank) V^T + 1e-4 G, the oracle runs Alg. 1
with the same Omega (Philox stream 3) and the same power iterations in FP64.  The library's spectral
error ||A - U U^T A||_2 must agree with the oracle's to 2%, U must be orthonormal, the leading
singular values must agree, and Eckart-Young must hold.  At the full size (A 262144 x 8192 FP32,
r = 300, q = 2) the properties that hold at any size are checked with an independent FP64/FP32
torch power method on the GPU.
"""
import numpy as np
import pytest
import torch

from oracle import rsvd as orsvd
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


@pytest.mark.parametrize("m,n,rank,r,q", [(4096, 1024, 60, 40, 2), (3000, 700, 30, 25, 0), (2048, 2048, 100, 75, 1)])
def test_rsvd_matches_oracle(rsk, m, n, rank, r, q):
    A = synthetic.lowrank_plus_noise(m, n, rank, seed=m + n, noise=1e-4, device="cpu")
    U, s, Vt = rsk.rsk_rsvd(A.cuda(), r, power_iters=q, zeta=8, seed=5)
    A64 = A.double().numpy()
    Ug = U.double().cpu().numpy()
    assert np.abs(Ug.T @ Ug - np.eye(r)).max() <= 1e-4
    e_gpu = orsvd.spectral_error(A64, Ug, iters=60, seed=1)
    Q = orsvd.range_finder(A64, r, q, zeta=8, seed=5)
    e_ref = orsvd.spectral_error(A64, Q, iters=60, seed=1)
    assert abs(e_gpu - e_ref) <= 0.02 * e_ref, (e_gpu, e_ref)
    sv = np.linalg.svd(A64, compute_uv=False)
    assert e_gpu >= sv[r] * (1 - 1e-6)                       # Eckart-Young
    _, s_ref, _ = orsvd.rsvd(A64, r, q, zeta=8, seed=5)
    sg = s.cpu().numpy()
    assert np.all(np.diff(sg) <= 1e-12)                     # descending
    assert np.allclose(sg[:10], s_ref[:10], rtol=1e-2)
    rec = (Ug * sg[None, :]) @ Vt.double().cpu().numpy()
    err_rec = np.linalg.norm(A64 - rec, 2)
    assert err_rec <= 1.05 * e_gpu + 1e-3 * sv[0]


def test_rsvd_invalid(rsk):
    A = torch.zeros(100, 50, device="cuda")
    with pytest.raises(rsk.RskError):
        rsk.rsk_rsvd(A, 60)                                 # r > min(m, n)
    with pytest.raises(rsk.RskError):
        rsk.rsk_rsvd(A, 4, zeta=8)                          # zeta > r
    with pytest.raises(rsk.RskError):
        rsk.rsk_rsvd(torch.zeros(1000, 500, device="cuda"), 321)   # r beyond the supported rank (320)


def _power_norm(apply, n, iters, gen):
    v = torch.randn(n, generator=gen, device="cuda", dtype=torch.float64)
    v /= v.norm()
    est = 0.0
    for _ in range(iters):
        y, v = apply(v)
        est = y.norm().item()
        v = v / v.norm()
    return est


def test_rsvd_full_size_properties(rsk):
    """A 262144 x 8192 FP32 = U diag(j^-2, j <= 400) V^T + 1e-4 G, r = 300, q = 2."""
    m, n, rank, r = 262144, 8192, 400, 300
    A = synthetic.lowrank_plus_noise(m, n, rank, seed=2025, noise=1e-4, device="cuda")
    U, s, Vt = rsk.rsk_rsvd(A, r, power_iters=2, zeta=8, seed=0)
    torch.cuda.synchronize()
    UtU = U.double().T @ U.double()
    assert (UtU - torch.eye(r, device="cuda", dtype=torch.float64)).abs().max().item() <= 1e-4
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    Ad = A.double()
    Ud = U.double()

    def resid(v):
        y = Ad @ v
        y = y - Ud @ (Ud.T @ y)
        return y, Ad.T @ y

    err = _power_norm(resid, n, 20, g)
    # Eckart-Young: ||A - Q Q^T A|| >= sigma_{r+1}(A) >= sigma_{r+1} of the noise-free part
    assert err >= (r + 1) ** -2.0
    # the noise floor ||1e-4 G||_2 ~ 1e-4 (sqrt(m) + sqrt(n)) bounds what any rank-r basis can reach;
    # q = 2 must land within a small factor of it
    floor = 1e-4 * (np.sqrt(m) + np.sqrt(n))
    assert err <= 2.0 * floor, (err, floor)
    sg = s.cpu().numpy()
    assert np.all(np.diff(sg) <= 1e-9)
    assert abs(sg[0] - 1.0) <= 0.05
