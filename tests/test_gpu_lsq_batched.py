"""GPU parity of the batched sketch-and-precondition solver (row a8).

Problems of uneven n_i and k_i (the batched workload's shape, scaled down): Gaussian A_i with column
scales logspaced over [1e-6, 1] in FP32 storage, Gaussian b_i.  Every x_i must have backward error
<= 1e-10 as recomputed by the oracle's FP64 code, in the mixed form (FP32 sketch, FP32 CG,
double-float residual passes) and in the all-FP64 form, and the batched solution must agree with
the single-problem solver run with the same seed.
"""
import numpy as np
import pytest
import torch

from oracle import lsq as olsq
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsk():
    import paper_2508_21189_gb300 as m
    return m


def make_batch(count, seed, n_lo=1024, n_hi=20000, k_lo=4, k_hi=64):
    ns, ks = synthetic.batched_sizes(count, seed, n_lo=n_lo, n_hi=n_hi, k_lo=k_lo, k_hi=k_hi)
    As, bs = [], []
    for i, (n, k) in enumerate(zip(ns, ks)):
        A, b = synthetic.batched_problem(n, k, seed=1000 * seed + i, device="cpu", dtype=torch.float32)
        As.append(A)
        bs.append(b)
    return As, bs


@pytest.mark.parametrize("sketch,inner", [(torch.float32, torch.float32), (torch.float64, torch.float64)])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
def test_batched_backward_error(rsk, sketch, inner, kind):
    # narrow: k_i <= 64 (the four-block column path); wide: k_i in [100, 256] (eight blocks)
    As, bs = make_batch(24, 3) if kind == "narrow" else make_batch(8, 5, n_lo=2000, n_hi=12000, k_lo=100, k_hi=256)
    xs, infos = rsk.rsk_lstsq_sketch_precond_batched([A.cuda() for A in As], [b.cuda() for b in bs],
                                                     sketch_dtype=sketch, inner_dtype=inner, seed=7)
    for A, b, x, info in zip(As, bs, xs, infos):
        A64, b64, x64 = A.double().numpy(), b.numpy(), x.cpu().numpy()
        eta = olsq.backward_error(A64, b64, x64)
        assert eta <= 1e-10, (eta, info)
        assert info["status"] == "RSK_OK"
        # the reported norms are those of the returned x: ||b - A x|| and ||A||_F
        rn = np.linalg.norm(b64 - A64 @ x64)
        assert abs(info["residual_norm"] - rn) <= 1e-5 * rn, (info["residual_norm"], rn)
        fn = np.linalg.norm(A64)
        assert abs(info["frobenius_norm"] - fn) <= 1e-5 * fn, (info["frobenius_norm"], fn)


@pytest.mark.parametrize("lo_exp", [-6.0, -10.0])
def test_batched_fp32_qr_preconditioner(rsk, lo_exp):
    # qr_dtype float32 factors [S A | S b] in FP32.  Householder QR is column-wise backward stable, so
    # for column-scaled A (scales 10^lo_exp .. 1) A R^{-1} stays well conditioned however small the
    # scales: with the same sketch and inner precision, the FP32-QR solve needs no more refinement steps
    # and CG iterations than the FP64-QR solve, up to a small slack, and reaches the same eta.
    ns, ks = synthetic.batched_sizes(10, 6, n_lo=2000, n_hi=16000, k_lo=16, k_hi=200)
    As, bs = [], []
    for i, (n, k) in enumerate(zip(ns, ks)):
        A, b = synthetic.batched_problem(n, k, seed=7000 + i, lo_exp=lo_exp, dtype=torch.float32)
        As.append(A.cuda())
        bs.append(b.cuda())
    runs = {}
    for sk in (torch.float32, torch.float64):
        for qr in (torch.float64, torch.float32):
            xs, infos = rsk.rsk_lstsq_sketch_precond_batched(As, bs, sketch_dtype=sk, inner_dtype=torch.float32,
                                                             qr_dtype=qr, seed=13)
            for A, b, x, info in zip(As, bs, xs, infos):
                eta = olsq.backward_error(A.double().cpu().numpy(), b.cpu().numpy(), x.cpu().numpy())
                assert eta <= 1e-10, (sk, qr, eta, info)
            runs[(sk, qr)] = infos
    for sk in (torch.float32, torch.float64):
        for info, r in zip(runs[(sk, torch.float32)], runs[(sk, torch.float64)]):
            assert info["refine_steps"] <= r["refine_steps"] + 2, (sk, info, r)
            assert info["inner_iters"] <= 2 * r["inner_iters"] + 20, (sk, info, r)


def test_batched_matches_single(rsk):
    As, bs = make_batch(6, 4)
    xs, _ = rsk.rsk_lstsq_sketch_precond_batched([A.cuda() for A in As], [b.cuda() for b in bs],
                                                 sketch_dtype=torch.float32, inner_dtype=torch.float32, seed=21)
    for i, (A, b, x) in enumerate(zip(As, bs, xs)):
        xi, _ = rsk.rsk_lstsq_sketch_precond(A.cuda(), b.cuda(), 4 * A.shape[1], seed=21 + i,
                                             sketch_dtype=torch.float32, inner_dtype=torch.float32)
        # both satisfy eta <= 1e-10; solutions agree to the conditioning of the problem
        rel = (x - xi).norm().item() / xi.norm().item()
        assert rel <= 1e-4, rel


@pytest.mark.parametrize("shapes,ds,zeta", [([(1, 1)], [1], 1),
                                            ([(5, 5), (3000, 1), (2049, 17), (4097, 3)], [16, 8, 68, 12], 4)])
def test_batched_edge_shapes(rsk, shapes, ds, zeta):
    # square (consistent) systems, k = 1, row counts one past a tile boundary
    g = torch.Generator().manual_seed(0)
    As = [torch.randn(n, k, generator=g, dtype=torch.float32) for n, k in shapes]
    bs = [torch.randn(A.shape[0], generator=g, dtype=torch.float64) for A in As]
    xs, infos = rsk.rsk_lstsq_sketch_precond_batched([A.cuda() for A in As], [b.cuda() for b in bs],
                                                     ds=ds, zeta=zeta, sketch_dtype=torch.float32,
                                                     inner_dtype=torch.float32, raise_on_nonconvergence=False)
    for A, b, x, info in zip(As, bs, xs, infos):
        assert info["status"] == "RSK_OK", info
        eta = olsq.backward_error(A.double().numpy(), b.numpy(), x.cpu().numpy())
        assert eta <= 1e-10, (eta, info)
        ref = np.linalg.lstsq(A.double().numpy(), b.numpy(), rcond=None)[0]
        assert np.allclose(x.cpu().numpy(), ref, rtol=1e-6, atol=1e-8)


def test_batched_invalid(rsk):
    A = torch.zeros(10, 300, device="cuda")       # k above the batched limit
    b = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(rsk.RskError):
        rsk.rsk_lstsq_sketch_precond_batched([A], [b])
    A = torch.zeros(100, 10, device="cuda")
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(rsk.RskError):   # the QR runs in FP64 or FP32 only
        rsk.rsk_lstsq_sketch_precond_batched([A], [b], qr_dtype=torch.bfloat16)


def test_batched_full_size_workload(rsk):
    """The benchmark's batched workload: 512 problems, n_i log-uniform in [4096, 262144], k_i uniform
    in [16, 256], Gaussian A_i x logspace(-6, 0) column scales in FP32, Gaussian b_i, d_i = 4 k_i;
    every eta <= 1e-10 recomputed independently in FP64 torch arithmetic."""
    ns, ks = synthetic.batched_sizes(512, seed=404)
    As, bs = [], []
    for i, (n, k) in enumerate(zip(ns, ks)):
        A, b = synthetic.batched_problem(n, k, seed=10_000 + i, device="cuda", dtype=torch.float32)
        As.append(A)
        bs.append(b)
    xs, infos = rsk.rsk_lstsq_sketch_precond_batched(As, bs, zeta=8, seed=9, sketch_dtype=torch.float32,
                                                     inner_dtype=torch.float32)
    worst = 0.0
    for A, b, x, info in zip(As, bs, xs, infos):
        A64, b64 = A.double(), b
        r = b64 - A64 @ x
        nr, fa = r.norm().item(), A64.norm().item()
        eta = min((A64.T @ r).norm().item() / (fa * nr), nr / (fa * x.norm().item() + b64.norm().item()))
        worst = max(worst, eta)
        assert info["status"] == "RSK_OK"
    assert worst <= 1e-10, worst
