"""Pins for the oracle's Philox generator and SparseUniform sketch (CPU only).

Each check is fixed by the paper's definition or by mathematics, not by re-running the
oracle's own formula: published Philox answers, the exact structure of Def. SparseUniform
(zeta distinct positions per column, values +-zeta^{-1/2}), uniformity of the sampled
subsets, the isotropy E[S^T S] = I of an oblivious subspace embedding (Sec. 2, Def. OSE/OSI),
and brute-force dense products.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import philox, sparse_sign

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10([v[0:4]], v[4:6])[0]
        assert [int(x) for x in out] == v[6:10]


def test_philox_word_layout():
    # word(seed, s, e, t) = philox(key=(seed_lo, seed_hi), ctr=(e_lo, e_hi, s, t>>2))[t & 3]
    seed = 0x0123456789ABCDEF
    e = 0x0000000500000007
    blk = philox.philox4x32_10([[7, 5, 3, 2]], [0x89ABCDEF, 0x01234567])[0]
    for t in range(8, 12):
        assert int(philox.words(seed, 3, e, t)) == int(blk[t & 3])


@pytest.mark.parametrize("n,d,zeta", [(1000, 17, 8), (3000, 400, 8), (500, 8, 8), (257, 33, 1), (300, 64, 32)])
def test_structure(n, d, zeta):
    rows, signs = sparse_sign.columns(n, d, zeta, seed=11)
    assert rows.shape == (n, zeta) and signs.shape == (n, zeta)
    assert rows.min() >= 0 and rows.max() < d
    srt = np.sort(rows, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0), "positions within a column must be distinct"
    assert set(np.unique(signs)) <= {-1, 1}
    S = sparse_sign.dense(min(n, 200), d, zeta, seed=11)
    nnz = (S != 0).sum(axis=0)
    assert np.all(nnz == zeta)
    # column norms are exactly one up to the rounding of zeta^{-1/2}
    assert np.allclose((S * S).sum(axis=0), 1.0, rtol=0, atol=4 * 2.0**-53 * zeta)
    # integer pattern: squared norms are exactly zeta
    assert np.all(((S != 0).astype(np.int64)).sum(axis=0) == zeta)


def test_floyd_subsets_uniform():
    # d = 5, zeta = 2: the 10 two-element subsets must be equally likely (Def. SparseUniform:
    # positions uniform without replacement).  Chi-square over 200k columns, 9 dof.
    n, d, zeta = 200_000, 5, 2
    rows, _ = sparse_sign.columns(n, d, zeta, seed=3)
    keys = np.sort(rows, axis=1)
    idx = {c: i for i, c in enumerate(itertools.combinations(range(d), zeta))}
    counts = np.zeros(len(idx))
    for a, b in keys:
        counts[idx[(a, b)]] += 1
    exp = n / len(idx)
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 27.9, chi2   # p = 0.001 quantile of chi^2_9


def test_marginals_and_pairs():
    # P(i in column j) = zeta/d, P(i, i' both in column j) = zeta(zeta-1)/(d(d-1)):
    # the indicator moments used in the SparseCol / CountSketch moment lemmas (App. C).
    n, d, zeta = 100_000, 16, 4
    rows, _ = sparse_sign.columns(n, d, zeta, seed=5)
    ind = np.zeros((n, d), dtype=np.float64)
    np.put_along_axis(ind, rows, 1.0, axis=1)
    p1 = ind.mean(axis=0)
    assert np.allclose(p1, zeta / d, atol=5 * np.sqrt(zeta / d / n))
    p2 = (ind.T @ ind) / n
    off = p2[~np.eye(d, dtype=bool)]
    target = zeta * (zeta - 1) / (d * (d - 1))
    assert np.allclose(off, target, atol=6 * np.sqrt(target / n))


def test_isotropy_monte_carlo():
    # E[S^T S] = I (each draw has S^T S diag == 1 exactly), E[S S^T] = (n/d) I.
    n, d, zeta, trials = 24, 12, 3, 3000
    StS = np.zeros((n, n))
    SSt = np.zeros((d, d))
    for s in range(trials):
        S = sparse_sign.dense(n, d, zeta, seed=1000 + s)
        StS += S.T @ S
        SSt += S @ S.T
    StS /= trials
    SSt /= trials
    assert np.allclose(np.diag(StS), 1.0, atol=1e-12)
    assert np.abs(StS - np.eye(n)).max() < 0.06
    assert np.abs(SSt - (n / d) * np.eye(d)).max() < 0.12


def test_signs_balanced():
    n, d, zeta = 50_000, 64, 8
    _, signs = sparse_sign.columns(n, d, zeta, seed=9)
    assert abs(signs.mean()) < 4 / np.sqrt(n * zeta)
    # independent across positions: E[s_q s_q'] = 0
    c = (signs[:, 0].astype(float) * signs[:, 7]).mean()
    assert abs(c) < 4 / np.sqrt(n)


def test_sign_bits_roundtrip():
    n, d, zeta = 100, 40, 8
    _, signs = sparse_sign.columns(n, d, zeta, seed=2)
    bits = sparse_sign.sign_bits(signs)
    j = np.arange(n, dtype=np.uint64)
    w = philox.words(2, 0, j, zeta).astype(np.uint64)
    mask = np.uint64((1 << zeta) - 1)
    assert np.array_equal(bits.astype(np.uint64), w & mask)


@pytest.mark.parametrize("n,d,zeta,k", [(64, 16, 8, 3), (256, 32, 4, 5), (100, 7, 7, 1)])
def test_apply_brute_force(n, d, zeta, k):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((n, k))
    S = sparse_sign.dense(n, d, zeta, seed=4)
    ref = np.zeros((d, k))
    for i in range(d):            # dense triple loop
        for c in range(k):
            acc = 0.0
            for j in range(n):
                acc += S[i, j] * A[j, c]
            ref[i, c] = acc
    out = sparse_sign.apply(A, d, zeta, seed=4)
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_csr_inverts_columns():
    n, d, zeta = 5000, 300, 8
    rowptr, cols, neg = sparse_sign.csr(n, d, zeta, seed=7)
    rows, signs = sparse_sign.columns(n, d, zeta, seed=7)
    assert rowptr[0] == 0 and rowptr[-1] == n * zeta
    rebuilt = {}
    for i in range(d):
        seg = cols[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(seg) > 0), "each row lists columns in ascending order"
        for j, ng in zip(seg, neg[rowptr[i]:rowptr[i + 1]]):
            rebuilt[(i, int(j))] = -1 if ng else 1
    for j in range(0, n, 37):
        for q in range(zeta):
            assert rebuilt[(int(rows[j, q]), j)] == signs[j, q]
    assert len(rebuilt) == n * zeta


def test_injectivity_dilation_coordinate_subspace():
    # The injectivity / dilation estimator of the paper's OSI experiment (Fig. 2, Sec. 1.5): the
    # adversarial orthonormal Q = [e_1 ... e_r] and embedding dimension 2r.  With zeta = 8 the sparse
    # embedding should behave like a 2r x r Gaussian, whose squared extreme singular values tend to
    # (1 -+ 1/sqrt 2)^2 (Marchenko-Pastur).  A missing zeta^{-1/2}, a repeated row within a column or
    # a wrong zeta moves them far outside 25 %.
    r = 200
    lo, hi = [], []
    for seed in range(5):
        SQ = sparse_sign.dense(r, 2 * r, 8, seed)   # S restricted to its first r columns
        sv = np.linalg.svd(SQ, compute_uv=False)
        lo.append(sv[-1] ** 2)
        hi.append(sv[0] ** 2)
    alpha, beta = (1 - 2 ** -0.5) ** 2, (1 + 2 ** -0.5) ** 2
    assert abs(np.median(lo) / alpha - 1) < 0.25, lo
    assert abs(np.median(hi) / beta - 1) < 0.25, hi
