"""The seeded input generators produce the workloads they are documented to produce.

CPU only: column scales of the column-scaled Gaussians, the exact singular values of the
least-squares matrix, the ranges and log-uniform / uniform laws of the uneven batch, and the
spectrum of the low-rank-plus-noise matrix.  These are the input recipes the benchmark and the
parity tests rely on.
"""
import math

import numpy as np
import torch

import synthetic


def test_seeded_and_deterministic():
    a = synthetic.gaussian(50, 7, seed=3)
    b = synthetic.gaussian(50, 7, seed=3)
    c = synthetic.gaussian(50, 7, seed=4)
    assert torch.equal(a, b)
    assert not torch.equal(a, c)


def test_colscaled_gaussian_column_scales():
    n, k = 40000, 16
    A = synthetic.colscaled_gaussian(n, k, seed=1, lo_exp=-3.0, hi_exp=0.0, dtype=torch.float32).double()
    scales = np.logspace(-3.0, 0.0, k)
    std = A.std(dim=0).numpy()
    # sample standard deviation of n Gaussians: relative error ~ 1 / sqrt(2 n) = 0.35%
    assert np.all(np.abs(std / scales - 1.0) < 0.02), std / scales
    assert abs(float(A.mean())) < 0.02


def test_lsq_problem_singular_values_and_noise():
    n, k = 600, 12
    A, b, x = synthetic.lsq_problem(n, k, seed=5, cond_exp=8.0, noise=1e-6)
    sv = np.linalg.svd(A.numpy(), compute_uv=False)
    expected = np.logspace(0.0, -8.0, k)
    # Q_U has orthonormal columns and V is orthogonal, so the singular values are sigma exactly
    # (up to FP64 rounding relative to sigma_1)
    assert np.allclose(sv, expected, rtol=0, atol=1e-13), sv
    r = (b - A @ x).numpy()
    assert 0.5e-6 * math.sqrt(n) < np.linalg.norm(r) < 1.5e-6 * math.sqrt(n)


def test_batched_sizes_laws():
    ns, ks = synthetic.batched_sizes(4000, seed=404)
    ns, ks = np.array(ns), np.array(ks)
    assert ns.min() >= 4096 and ns.max() <= 262144
    assert ks.min() >= 16 and ks.max() <= 256
    # log-uniform n: log(n / 4096) / log(64) uniform on [0, 1): mean 1/2, variance 1/12
    u = np.log(ns / 4096.0) / np.log(64.0)
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1.0 / 12.0) < 0.01
    # uniform integer k on [16, 256]: mean 136
    assert abs(ks.mean() - 136.0) < 4.0
    assert len(np.unique(ks)) > 200


def test_batched_problem_column_scales():
    A, b = synthetic.batched_problem(30000, 8, seed=11, lo_exp=-6.0, dtype=torch.float64)
    std = A.std(dim=0).numpy()
    assert np.all(np.abs(std / np.logspace(-6.0, 0.0, 8) - 1.0) < 0.03)
    assert abs(float(b.std()) - 1.0) < 0.03


def test_lowrank_plus_noise_spectrum():
    m, n, rank = 3000, 400, 30
    A = synthetic.lowrank_plus_noise(m, n, rank, seed=2, noise=0.0).double().numpy()
    sv = np.linalg.svd(A, compute_uv=False)
    j = np.arange(1, rank + 1)
    # orthonormalised U, V: the leading singular values are j^-2 (FP32 generation), the rest zero
    assert np.allclose(sv[:rank], j ** -2.0, rtol=1e-4), sv[:rank]
    assert sv[rank] < 1e-5
    B = synthetic.lowrank_plus_noise(m, n, rank, seed=2, noise=1e-4).double().numpy()
    # the noise adds about 1e-4 (sqrt(m) + sqrt(n)) to the spectral norm of the tail
    tail = np.linalg.svd(B, compute_uv=False)[rank + 5]
    assert 0.3e-4 * (math.sqrt(m) + math.sqrt(n)) < tail < 1.2e-4 * (math.sqrt(m) + math.sqrt(n))
