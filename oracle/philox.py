"""Philox4x32-10 counter-based generator, written from its published definition.

Reference: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11, Sec. 3 (the Philox S-box and key schedule).
The multipliers and the Weyl key increments below are the ones that paper gives for
the 4x32 variant; 10 rounds is the variant the paper recommends.

The paper under study (arxiv 2508.21189) only asks for iid Rademacher signs and for
positions sampled uniformly without replacement (Def. "SparseUniform", Sec. 3.2.1);
it does not fix a generator.  This stream layout is the reading used on both sides:

    word(seed, stream, entity, t) = Philox4x32-10(
        key = (seed_lo, seed_hi),
        ctr = (entity_lo, entity_hi, stream, t >> 2))[t & 3]

Pinned against the published known-answer vectors (tests/golden/philox_kat.txt).
TEST INFRASTRUCTURE: part of the oracle; see oracle/__init__.py.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """Apply ten Philox rounds to counters ``ctr`` (N x 4, uint32) under ``key`` (N x 2 or 2).

    One round: multiply words 0 and 2 by the two constants (full 64-bit products),
    then the new block is (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)).
    The key is bumped by the Weyl constants between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint64)
    if k.ndim == 1:
        k = np.broadcast_to(k, (c.shape[0], 2))
    x0, x1, x2, x3 = (c[:, i].copy() for i in range(4))
    k0 = k[:, 0].copy()
    k1 = k[:, 1].copy()
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = x0 * M0
        p1 = x2 * M1
        hi0, lo0 = p0 >> S32, p0 & MASK32
        hi1, lo1 = p1 >> S32, p1 & MASK32
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=1).astype(np.uint32)


def words(seed, stream, entity, t):
    """Vectorised ``word(seed, stream, entity, t)``; entity and t broadcast together."""
    entity = np.asarray(entity, dtype=np.uint64)
    t = np.asarray(t, dtype=np.uint64)
    entity, t = np.broadcast_arrays(entity, t)
    shape = entity.shape
    e = entity.reshape(-1)
    tt = t.reshape(-1)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)
    ctr = np.stack([e & MASK32, e >> S32,
                    np.full(e.shape, stream, dtype=np.uint64), tt >> np.uint64(2)], axis=1)
    out = philox4x32_10(ctr, key)
    sel = (tt & np.uint64(3)).astype(np.int64)
    return out[np.arange(out.shape[0]), sel].reshape(shape)
