"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle's callers.  It holds no
arithmetic of the sketching method itself: only random test matrices and right-hand sides.
Every generator is deterministic given (seed, device).  CPU and CUDA torch generators give
different streams, so a test draws its inputs once and hands the same values to both sides.
"""
import math

import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian(n, k, seed, device="cpu", dtype=torch.float64):
    """n x k matrix of iid N(0, 1) entries."""
    return torch.randn(n, k, generator=_gen(seed, device), device=device, dtype=dtype)


def colscaled_gaussian(n, k, seed, lo_exp=-3.0, hi_exp=0.0, device="cpu", dtype=torch.float32):
    """N(0,1) entries times per-column scales logspaced over [10^lo_exp, 10^hi_exp].

    The embedding-throughput workload: A 2^22 x 256 with scales logspaced over [1e-3, 1].
    Generated in float32 and cast, so BF16 / FP32 inputs of one seed hold the same values
    up to the final rounding.
    """
    g = _gen(seed, device)
    A = torch.randn(n, k, generator=g, device=device, dtype=torch.float32)
    s = torch.logspace(lo_exp, hi_exp, k, device=device, dtype=torch.float32)
    A.mul_(s[None, :])
    return A.to(dtype)


def lsq_problem(n, k, seed, cond_exp=8.0, noise=1e-6, device="cpu"):
    """A = Q_U diag(sigma) V^T (n x k, FP64), sigma logspaced from 1 to 10^-cond_exp;
    b = A x* + noise * N(0, 1), x* ~ N(0, I).  Returns (A, b, x_true)."""
    g = _gen(seed, device)
    G = torch.randn(n, k, generator=g, device=device, dtype=torch.float64)
    QU, _ = torch.linalg.qr(G)
    del G
    H = torch.randn(k, k, generator=g, device=device, dtype=torch.float64)
    V, Rv = torch.linalg.qr(H)
    V = V * torch.sign(torch.diagonal(Rv))[None, :]
    sigma = torch.logspace(0.0, -cond_exp, k, device=device, dtype=torch.float64)
    A = QU.mul_(sigma[None, :]) @ V.T
    x = torch.randn(k, generator=g, device=device, dtype=torch.float64)
    b = A @ x + noise * torch.randn(n, generator=g, device=device, dtype=torch.float64)
    return A, b, x


def batched_sizes(count, seed, n_lo=4096, n_hi=262144, k_lo=16, k_hi=256):
    """Uneven batch shapes: n_i log-uniform in [n_lo, n_hi], k_i uniform in [k_lo, k_hi]."""
    g = _gen(seed, "cpu")
    u = torch.rand(count, generator=g, dtype=torch.float64)
    v = torch.rand(count, generator=g, dtype=torch.float64)
    ns = [int(n_lo * (n_hi / n_lo) ** float(ui)) for ui in u]
    ks = [k_lo + int((k_hi - k_lo + 1) * float(vi)) for vi in v]
    ks = [min(k, k_hi) for k in ks]
    return ns, ks


def batched_problem(n, k, seed, lo_exp=-6.0, device="cpu", dtype=torch.float32):
    """One problem of the uneven batch: Gaussian A with column scales logspaced over
    [10^lo_exp, 1] and Gaussian b."""
    g = _gen(seed, device)
    A = torch.randn(n, k, generator=g, device=device, dtype=torch.float64)
    A.mul_(torch.logspace(lo_exp, 0.0, k, device=device, dtype=torch.float64)[None, :])
    b = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    return A.to(dtype), b


def lowrank_plus_noise(m, n, rank, seed, noise=1e-4, decay=2.0, device="cpu",
                       dtype=torch.float32):
    """U diag(j^-decay, j <= rank) V^T + noise * G with U, V orthonormalised Gaussians."""
    g = _gen(seed, device)
    U, _ = torch.linalg.qr(torch.randn(m, rank, generator=g, device=device, dtype=torch.float32))
    V, _ = torch.linalg.qr(torch.randn(n, rank, generator=g, device=device, dtype=torch.float32))
    s = torch.arange(1, rank + 1, device=device, dtype=torch.float32).pow(-decay)
    A = (U * s[None, :]) @ V.T
    if noise:
        A.add_(torch.randn(m, n, generator=g, device=device, dtype=torch.float32), alpha=noise)
    return A.to(dtype)


def log2(n):
    return int(round(math.log2(n)))
