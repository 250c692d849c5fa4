"""Pins for the oracle's least-squares and RSVD pipelines (CPU only)."""
import numpy as np
import pytest

from oracle import lsq, rsvd, sparse_sign


def test_lstsq_k1_closed_form():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(3000)
    b = rng.standard_normal(3000)
    x, info = lsq.sketch_precond(a[:, None], b, d=8, zeta=4, seed=1)
    assert np.allclose(x[0], a @ b / (a @ a), rtol=1e-12)
    assert info["backward_err"] <= 1e-10


def test_lstsq_orthonormal_columns():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((4000, 20)))
    b = rng.standard_normal(4000)
    x, info = lsq.sketch_precond(Q, b, d=80, zeta=8, seed=2)
    assert np.allclose(x, Q.T @ b, atol=1e-11)
    assert np.allclose(lsq.exact(Q, b), Q.T @ b, atol=1e-12)


def test_lstsq_consistent_system():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((5000, 30)) * np.logspace(-4, 0, 30)[None, :]
    xt = rng.standard_normal(30)
    b = A @ xt
    x, info = lsq.sketch_precond(A, b, d=120, zeta=8, seed=3)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    assert np.allclose(x, xt, rtol=1e-6, atol=1e-6)


def test_lstsq_ill_conditioned_matches_lapack():
    rng = np.random.default_rng(3)
    n, k = 20000, 50
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    A = (U * np.logspace(0, -8, k)[None, :]) @ V.T
    xt = rng.standard_normal(k)
    b = A @ xt + 1e-6 * rng.standard_normal(n)
    x, info = lsq.sketch_precond(A, b, d=4 * k, zeta=8, seed=4)
    assert info["backward_err"] <= 1e-10
    xs = np.linalg.lstsq(A, b, rcond=None)[0]      # SVD-based LAPACK solver
    assert lsq.backward_error(A, b, xs) <= 1e-10
    # both are minimisers: residual norms agree to the conditioning of the residual
    rn = np.linalg.norm(b - A @ x)
    rs = np.linalg.norm(b - A @ xs)
    assert abs(rn - rs) <= 1e-9 * rs


def test_backward_error_detects_perturbation():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((2000, 10))
    b = rng.standard_normal(2000)
    xs = lsq.exact(A, b)
    assert lsq.backward_error(A, b, xs) < 1e-14
    assert lsq.backward_error(A, b, xs + 1e-3) > 1e-5
    # definition (inconsistent problem: the normal-equation term is the smaller one)
    x1 = xs + 1e-3
    r = b - A @ x1
    fa = np.sqrt((A ** 2).sum())
    ls = np.sqrt(((A.T @ r) ** 2).sum()) / (fa * np.sqrt((r ** 2).sum()))
    cons = np.sqrt((r ** 2).sum()) / (fa * np.sqrt((x1 ** 2).sum()) + np.sqrt((b ** 2).sum()))
    assert ls < cons
    assert np.isclose(lsq.backward_error(A, b, x1), ls, rtol=1e-12)


def test_backward_error_consistent_system():
    # a square nonsingular system solved exactly: r is pure rounding, eta must be tiny
    rng = np.random.default_rng(9)
    A = rng.standard_normal((6, 6))
    b = rng.standard_normal(6)
    x = np.linalg.solve(A, b)
    assert lsq.backward_error(A, b, x) < 1e-13
    assert lsq.backward_error(A, b, x + 1e-6) > 1e-9


def test_lsqr_unpreconditioned_small():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((300, 12))
    y = rng.standard_normal(300)
    z, its = lsq.lsqr(lambda v: M @ v, lambda u: M.T @ u, y, 12, 1e-14, 200)
    assert np.allclose(z, np.linalg.lstsq(M, y, rcond=None)[0], atol=1e-10)


def test_rsvd_exact_low_rank():
    rng = np.random.default_rng(6)
    m, n, rank = 400, 300, 5
    A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    U, s, Vt = rsvd.rsvd(A, r=12, power_iters=0, zeta=4, seed=1)
    assert np.allclose((U * s) @ Vt, A, atol=1e-9 * np.abs(A).max())
    assert np.allclose(s[:rank], np.linalg.svd(A, compute_uv=False)[:rank], rtol=1e-10)


def test_rsvd_error_bounds():
    rng = np.random.default_rng(7)
    m, n, r = 600, 400, 20
    Ua, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Va, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.arange(1, n + 1, dtype=float) ** -2.0
    A = (Ua * sig[None, :]) @ Va.T
    Q = rsvd.range_finder(A, r, 2, zeta=8, seed=3)
    true = np.linalg.norm(A - Q @ (Q.T @ A), 2)
    est = rsvd.spectral_error(A, Q, iters=60, seed=0)
    assert est <= true * (1 + 1e-12) and est >= 0.99 * true      # power method pin
    assert true >= sig[r] * (1 - 1e-10)                          # Eckart-Young
    assert true <= 5 * sig[r]                                    # q = 2 power iterations


def test_omega_rows_sparse():
    Om = rsvd.omega(500, 30, 8, seed=2)
    assert np.all((Om != 0).sum(axis=1) == 8)
    assert np.allclose(np.abs(Om[Om != 0]), 1 / np.sqrt(8))
    # same pattern as the left sparse sign drawn from stream 3
    S = sparse_sign.dense(500, 30, 8, seed=2, stream=sparse_sign.STREAM_RSVD)
    assert np.array_equal(Om, S.T)


def test_sketch_and_solve_residual_bound():
    # Sketch-and-solve with an OSI (Sec. 2.3, theorem on sketch-and-solve): with probability >= 9/10
    # the warm start's squared residual is within C / alpha of the optimum.  With d = 4k the
    # injectivity is about (1 - sqrt(k/d))^2 = 1/4; the check takes C = 1 (a bound of 4) on 10 seeds
    # and requires 9 to pass, and every ratio to be >= 1 (the exact solution is optimal).
    g = np.random.default_rng(1)
    ratios = []
    for seed in range(10):
        n, k = 4000, 20
        A = g.standard_normal((n, k))
        b = g.standard_normal(n)
        _, info = lsq.sketch_precond(A, b, 4 * k, 8, seed, max_refine=0)
        xs = lsq.exact(A, b)
        r0 = np.linalg.norm(A @ info["x0"] - b) ** 2
        rs = np.linalg.norm(A @ xs - b) ** 2
        ratios.append(r0 / rs)
    assert min(ratios) >= 1 - 1e-12, ratios
    assert sum(r <= 4.0 for r in ratios) >= 9, ratios


@pytest.mark.parametrize("q", [0, 1])
def test_rsvd_error_close_to_gaussian_test_matrix(q):
    # The paper's RSVD comparison (Sec. 1.4, Fig. 1): a sparse test matrix gives about the error of
    # a Gaussian one.  Baseline written here with numpy (Gaussian Omega, QR after every product);
    # the medians over 5 seeds must agree to 25 % and both must respect Eckart-Young.
    import synthetic
    A = synthetic.lowrank_plus_noise(3000, 600, 60, seed=7, noise=1e-3, device="cpu").double().numpy()
    r = 40
    sv = np.linalg.svd(A, compute_uv=False)
    es, eg = [], []
    for seed in range(5):
        Q = rsvd.range_finder(A, r, q, zeta=8, seed=seed)
        es.append(rsvd.spectral_error(A, Q, iters=60, seed=1))
        g = np.random.default_rng(100 + seed)
        Qg, _ = np.linalg.qr(A @ g.standard_normal((A.shape[1], r)))
        for _ in range(q):
            Qg, _ = np.linalg.qr(A.T @ Qg)
            Qg, _ = np.linalg.qr(A @ Qg)
        eg.append(np.linalg.norm(A - Qg @ (Qg.T @ A), 2))
    assert min(es) >= sv[r] * (1 - 1e-6) and min(eg) >= sv[r] * (1 - 1e-6)
    assert abs(np.median(es) / np.median(eg) - 1) < 0.25, (es, eg)
