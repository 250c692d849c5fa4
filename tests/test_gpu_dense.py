"""GPU checks of the dense steps of the low-rank algorithms (svd_econ, qr_econ) against LAPACK.

svd_econ: singular values within 8 q u_32 ||A||_2 of LAPACK's (one-sided Jacobi is accurate to a
small multiple of u relative to ||A||), V orthonormal to 1e-5, the columns of U whose singular value
exceeds 1e-2 ||A|| orthonormal to 1e-5, U diag(s) V^T = A to 1e-5 ||A||.  qr_econ: Q^T Q = I to
1e-5 even for kappa(X) = 1e5 (the Gram is accumulated in FP64), Q R = X to 1e-5 ||X||, R upper
triangular.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


def colmajor(A):
    return torch.from_numpy(np.asarray(A, dtype=np.float32)).cuda().t().contiguous().t()


def spectrum_matrix(m, q, decay, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, q)))
    V, _ = np.linalg.qr(rng.standard_normal((q, q)))
    s = decay ** np.arange(q) if decay < 1 else np.linspace(1, 2, q)
    return (U * s) @ V.T


@pytest.mark.parametrize("m,q,decay,seed", [(1, 1, 2.0, 0), (5, 3, 2.0, 1), (64, 64, 0.9, 2), (300, 300, 0.97, 3),
                                            (450, 300, 0.99, 4), (1000, 37, 0.5, 5), (2048, 512, 2.0, 6),
                                            (320, 304, 0.95, 7)])
def test_svd_econ_matches_lapack(rsk, m, q, decay, seed):
    A = spectrum_matrix(m, q, decay, seed).astype(np.float32).astype(np.float64)
    U, s, V = rsk.rsk_svd_econ(colmajor(A))
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    U, s, V = U.double().cpu().numpy(), s.double().cpu().numpy(), V.double().cpu().numpy()
    ref = np.linalg.svd(A, compute_uv=False)
    nrm = ref[0]
    assert np.all(np.diff(s) <= 0)
    assert np.abs(s - ref).max() <= 8 * q * U32 * nrm + 1e-30
    # left singular vectors are determined (and orthonormal) to ~u ||A|| / s_i: check those with
    # s_i > 1e-2 ||A||; V is a product of rotations and orthonormal throughout
    keep = s > 1e-2 * nrm
    Uk = U[:, keep]
    assert np.abs(Uk.T @ Uk - np.eye(Uk.shape[1])).max() <= 1e-5 * max(1, q / 100)
    assert np.abs(V.T @ V - np.eye(q)).max() <= 1e-5 * max(1, q / 100)
    assert np.abs((U * s) @ V.T - A).max() <= 1e-5 * nrm * max(1, q / 100)


@pytest.mark.parametrize("m,q,cond_exp,seed", [(1, 1, 0, 0), (100, 10, 0, 1), (5000, 64, 3, 2), (20000, 300, 5, 3),
                                               (4096, 330, 2, 4)])
def test_qr_econ_orthonormal(rsk, m, q, cond_exp, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, q))
    Qx, _ = np.linalg.qr(G)
    V, _ = np.linalg.qr(rng.standard_normal((q, q)))
    X = ((Qx * np.logspace(0, -cond_exp, q)) @ V.T).astype(np.float32).astype(np.float64)
    Q, R = rsk.rsk_qr_econ(colmajor(X))
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    Q, R = Q.double().cpu().numpy(), R.double().cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(q)).max() <= 1e-5
    assert np.allclose(np.tril(R, -1), 0)
    assert np.abs(Q @ R - X).max() <= 1e-5 * np.linalg.norm(X, 2)


@pytest.mark.parametrize("q,cond_exp,shift", [(1, 0, 0.0), (17, 1, 0.0), (300, 3, 0.0), (320, 2, 3e-5), (330, 1, 0.0),
                                               (100, 6, 3e-5)])
def test_cholesky_matches_lapack(rsk, q, cond_exp, shift):
    """R^T R = G + shift trace(G) I: R matches LAPACK's factor of the same FP32 matrix to FP32 accuracy
    (relative to the factor's norm, times the condition number)."""
    rng = np.random.default_rng(q)
    Vq, _ = np.linalg.qr(rng.standard_normal((q, q)))
    G = ((Vq * np.logspace(0, -cond_exp, q)) @ Vq.T).astype(np.float32).astype(np.float64)
    G = 0.5 * (G + G.T)
    R = rsk.rsk_cholesky(colmajor(G), shift_coeff=shift)
    torch.cuda.synchronize()
    rsk.rsk_sync_status()
    R = R.double().cpu().numpy()
    Gs = G + np.float32(shift) * np.float32(np.trace(G.astype(np.float32))) * np.eye(q)
    ref = np.linalg.cholesky(Gs).T
    assert np.allclose(np.tril(R, -1), 0)
    assert np.abs(R.T @ R - Gs).max() <= 64 * q * U32 * np.abs(Gs).max()
    assert np.abs(R - ref).max() <= 1e-5 * 10 ** cond_exp * np.abs(ref).max() * max(1, q / 64)


def test_cholesky_not_psd(rsk):
    G = np.eye(40)
    G[7, 7] = -1.0
    rsk.rsk_cholesky(colmajor(G))
    torch.cuda.synchronize()
    with pytest.raises(rsk.RskError):
        rsk.rsk_sync_status()


@pytest.mark.parametrize("q", [1, 31, 32, 33, 300, 330, 880])
def test_trinv_matches_solve(rsk, q):
    rng = np.random.default_rng(q + 1)
    # well conditioned: unit-order diagonal, off-diagonal entries of size q^-1/2 (kappa ~ 10)
    R = np.triu(rng.standard_normal((q, q)), 1) / (2 * q ** 0.5) + np.diag(1.0 + rng.random(q))
    R = R.astype(np.float32).astype(np.float64)
    Ri = rsk.rsk_trinv(colmajor(R))
    torch.cuda.synchronize()
    Ri = Ri.double().cpu().numpy()
    assert np.allclose(np.tril(Ri, -1), 0)
    assert np.abs(R @ Ri - np.eye(q)).max() <= 1e-5 * max(1, q / 64)
