"""GPU parity of the Nystrom approximation of a psd matrix (Alg. 2) against the FP64 oracle.

Both sides take the same test matrix (the library's sparse sketch, drawn from the same seed) and the
same shift rule.  The approximations A_hat = U diag(lambda) U^T are compared in the spectral norm:
||A_hat_gpu - A_hat_oracle||_2 <= max(1e-4 ||A||_2, 20 nu) (FP32 sketches and dense steps against
FP64; nu = sqrt(n) u ||Y||_F is the scale the shifted FP32 computation resolves), and the eigenvalues
agree to the same bound.  On a rank-20 psd matrix the error equals the FP64 oracle's, and U has
orthonormal columns.
"""
import numpy as np
import pytest
import torch

from oracle import nystrom as ony

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


def psd_matrix(n, decay, seed, rank=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = decay ** np.arange(n)
    if rank is not None:
        lam[rank:] = 0
    A = ((Q * lam) @ Q.T).astype(np.float32).astype(np.float64)
    return 0.5 * (A + A.T), lam


@pytest.mark.parametrize("kind", ["stack", "uniform"])
@pytest.mark.parametrize("n,k,rank,zeta,decay", [(64, 8, 8, 4, 0.7), (1000, 64, 40, 4, 0.9), (3000, 128, 128, 8, 0.97),
                                                 (2500, 300, 250, 4, 0.99)])
def test_parity_with_oracle(rsk, kind, n, k, rank, zeta, decay):
    A, _ = psd_matrix(n, decay, n + k)
    U, lam = rsk.rsk_nystrom_psd(torch.from_numpy(A.astype(np.float32)).cuda(), k, rank=rank, zeta=zeta, seed=5,
                                 kind=kind)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    U, lam = U.double().cpu().numpy(), lam.double().cpu().numpy()
    kd = {"uniform": 0, "stack": 1}[kind]
    Uo, lo = ony.psd_nystrom(A, k, zeta, 5, kind=kd, rank=rank)
    nA = np.linalg.norm(A, 2)
    # the FP32 computation resolves the spectrum to the shift's scale nu = sqrt(n) u ||Y||_F (the shifted
    # core Omega^T Y_nu has condition ~ ||A|| / nu): both sides use the same nu
    nu = np.sqrt(n) * ony.EPS32 * np.linalg.norm(A @ ony.test_matrix(n, k, zeta, 5, kd))
    tol = max(1e-4 * nA, 20 * nu)
    assert np.abs(U.T @ U - np.eye(rank)).max() <= 1e-4
    assert np.abs(lam - lo).max() <= tol
    assert np.linalg.norm((U * lam) @ U.T - (Uo * lo) @ Uo.T, 2) <= tol


def test_low_rank_recovery(rsk):
    A, _ = psd_matrix(2000, 0.8, 9, rank=20)
    U, lam = rsk.rsk_nystrom_psd(torch.from_numpy(A.astype(np.float32)).cuda(), 64, zeta=4, seed=2)
    U, lam = U.double().cpu().numpy(), lam.double().cpu().numpy()
    # the shifted Nystrom approximation of a rank-20 matrix: its error is the oracle's (FP64, same nu)
    Uo, lo = ony.psd_nystrom(A, 64, 4, 2, kind=1)
    err, err_o = np.linalg.norm(A - (U * lam) @ U.T, 2), np.linalg.norm(A - (Uo * lo) @ Uo.T, 2)
    assert err <= 1.1 * err_o + 1e-5 and err <= 1e-3 * np.linalg.norm(A, 2)
    assert np.all(lam[20:] <= 1e-4)


def test_rejects_bad_arguments(rsk):
    A = torch.eye(100, device="cuda")
    with pytest.raises(Exception):
        rsk.rsk_nystrom_psd(A, 30, zeta=4)          # SparseStack needs k % zeta == 0
    with pytest.raises(Exception):
        rsk.rsk_nystrom_psd(A, 400)                 # k > n


def lowrank_noise(n, d, r, seed, noise):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    V, _ = np.linalg.qr(rng.standard_normal((d, r)))
    A = (U * 0.8 ** np.arange(r)) @ V.T + noise * rng.standard_normal((n, d)) / np.sqrt(max(n, d))
    return A.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("kind", ["stack", "uniform"])
@pytest.mark.parametrize("n,d,k,p,zeta", [(500, 300, 16, 24, 4), (3000, 2000, 64, 96, 4), (6000, 5000, 200, 304, 8)])
def test_generalized_parity_with_oracle(rsk, kind, n, d, k, p, zeta):
    # generalized Nystrom (Algs. 4 and 5) against the FP64 oracle with the same test matrices:
    # both forms approximate A as well as the oracle does (same error to 1e-3 of ||A||), and agree
    # with the oracle's approximation to 1e-3 ||A||
    A = lowrank_noise(n, d, 40, n + d, 1e-3)
    kd = {"uniform": 0, "stack": 1}[kind]
    At = torch.from_numpy(A.astype(np.float32)).cuda()
    F, G, r = rsk.rsk_gen_nystrom(At, k, p=p, zeta=zeta, seed=3, kind=kind, form="outer")
    U, s, V, r5 = rsk.rsk_gen_nystrom(At, k, p=p, zeta=zeta, seed=3, kind=kind, form="svd")
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    F, G = F.double().cpu().numpy(), G.double().cpu().numpy()
    U, s, V = U.double().cpu().numpy(), s.double().cpu().numpy(), V.double().cpu().numpy()
    Fo, Go, ro = ony.gen_nystrom_outer(A, k, p, zeta, 3, kind=kd)
    Uo, so, Vo, r5o = ony.gen_nystrom_svd(A, k, p, zeta, 3, kind=kd)
    nA = np.linalg.norm(A, 2)
    ref4, ref5 = Fo @ Go.T, (Uo * so) @ Vo.T
    assert r == ro and r5 == r5o
    assert np.linalg.norm(F @ G.T - ref4, 2) <= 1e-3 * nA
    assert np.linalg.norm((U * s) @ V.T - ref5, 2) <= 1e-3 * nA
    assert abs(np.linalg.norm(A - F @ G.T, 2) - np.linalg.norm(A - ref4, 2)) <= 1e-3 * nA
    assert np.abs(s - so).max() <= 1e-3 * nA
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-4 and np.abs(V.T @ V - np.eye(k)).max() <= 1e-4
