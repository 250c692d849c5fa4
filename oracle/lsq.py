"""Least squares by sketch-and-precondition, plus the exact FP64 solution and backward error.

Paper: Alg. 3 (sketch-and-solve, Sec. 2.3) forms the sketched problem Psi^T A, Psi^T b and
solves it through a decomposition of the sketch; the paper names sketch-and-precondition
(Rokhlin-Tygert, Avron-Maymounkov-Toledo) as the standard route to high accuracy (Remark
after Cor. 2.x, Sec. 2.3) without spelling it out.  The steps used here:

  L1  Ahat = S A, bhat = S b with the same sparse sign S (oracle.sparse_sign).
  L2  Householder QR  Ahat = Q R  (LAPACK geqrf via numpy), signs fixed so diag(R) > 0.
  L3  warm start x0 = R^{-1} Q^T bhat  (Alg. 3 with a QR in place of the SVD: Ahat has
      full column rank for an embedding).
  L4  refinement: r = b - A x; stop when eta(x) <= tol; otherwise run LSQR (Paige &
      Saunders, ACM TOMS 1982) on min ||A R^{-1} z - r|| from z = 0 and set x += R^{-1} z.
  L5  eta(x) = min( ||A^T r||_2 / (||A||_F ||r||_2),  ||r||_2 / (||A||_F ||x||_2 + ||b||_2) ),
      r = b - A x, all in FP64: the two quantities of Paige & Saunders' LSQR stopping rules (S2 for
      least-squares problems, S1 for consistent ones).  For an inconsistent problem the first term
      governs; for a (nearly) consistent one r is rounding noise, the first term is a quotient of
      rounding errors and the second, the normwise backward error of A x = b, is the meaningful one.

The oracle runs every step in FP64.
TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np
import scipy.linalg as sla

from . import sparse_sign


def backward_error(A, b, x):
    """eta(x) = min(||A^T r|| / (||A||_F ||r||), ||r|| / (||A||_F ||x|| + ||b||)), r = b - A x (L5)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    r = b - A @ x
    fa = np.linalg.norm(A)
    nr = np.linalg.norm(r)
    if nr == 0.0:
        return 0.0
    ls = np.linalg.norm(A.T @ r) / (fa * nr)
    cons = nr / (fa * np.linalg.norm(x) + np.linalg.norm(b))
    return float(min(ls, cons))


def exact(A, b):
    """x* = argmin ||A x - b|| by Householder QR of the full A (FP64)."""
    Q, R = np.linalg.qr(np.asarray(A, dtype=np.float64), mode="reduced")
    return sla.solve_triangular(R, Q.T @ np.asarray(b, dtype=np.float64), lower=False)


def qr_r_positive(M):
    """Householder QR of M with diag(R) > 0; returns (Q, R)."""
    Q, R = np.linalg.qr(np.asarray(M, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def lsqr(matvec, rmatvec, rhs, k, tol, max_iters):
    """LSQR (Paige & Saunders 1982, Sec. 4) for min ||M z - rhs|| from z = 0.

    Stops when the estimate ||M^T rho|| <= tol * ||M||_F * ||rho|| (their stopping rule S2
    with ||M||_F estimated from the bidiagonal) or after max_iters steps.
    Returns (z, iterations).
    """
    u = np.array(rhs, dtype=np.float64, copy=True)
    beta = np.linalg.norm(u)
    z = np.zeros(k)
    if beta == 0.0:
        return z, 0
    u /= beta
    v = rmatvec(u)
    alpha = np.linalg.norm(v)
    if alpha == 0.0:
        return z, 0
    v /= alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = alpha * alpha
    it = 0
    for it in range(1, max_iters + 1):
        u = matvec(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u /= beta
        anorm2 += beta * beta
        v = rmatvec(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0:
            v /= alpha
        anorm2 += alpha * alpha
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        z = z + (phi / rho) * w
        w = v - (theta / rho) * w
        # ||M^T rho_it|| = phibar * alpha * |c|, ||rho_it|| = phibar
        if phibar * alpha * abs(c) <= tol * np.sqrt(anorm2) * phibar:
            break
    return z, it


def sketch_precond(A, b, d, zeta, seed, tol=1e-10, max_refine=10, inner_tol=1e-12,
                   max_inner=200):
    """Steps L1-L5 in FP64. Returns (x, info dict)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n, k = A.shape
    Ab = np.concatenate([A, b[:, None]], axis=1)
    SAb = sparse_sign.apply(Ab, d, zeta, seed)          # L1
    Q, R = qr_r_positive(SAb[:, :k])                    # L2
    x = sla.solve_triangular(R, Q.T @ SAb[:, k], lower=False)   # L3
    inner_total = 0
    steps = 0
    eta = backward_error(A, b, x)
    for steps in range(max_refine + 1):                 # L4
        if eta <= tol or steps == max_refine:
            break
        r = b - A @ x
        Rinv = lambda y: sla.solve_triangular(R, y, lower=False)
        RinvT = lambda y: sla.solve_triangular(R, y, lower=False, trans="T")
        z, its = lsqr(lambda v: A @ Rinv(v), lambda u: RinvT(A.T @ u), r, k, inner_tol, max_inner)
        inner_total += its
        x = x + Rinv(z)
        eta = backward_error(A, b, x)
    return x, {"backward_err": eta, "refine_steps": steps, "inner_iters": inner_total,
               "R": R, "x0": sla.solve_triangular(R, Q.T @ SAb[:, k], lower=False)}
