"""Philox4x32-10 counter-based generator, written from its published definition.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg, never by the product path.

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3 / Philox-4x32): a 128-bit counter (c0, c1, c2, c3) and a
64-bit key (k0, k1).  One round multiplies c0 and c2 by the constants
M0 = 0xD2511F53 and M1 = 0xCD9E8D57 into 64-bit products (hi, lo) and permutes:

    (c0, c1, c2, c3) <- (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),
                         hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

Between rounds the key is bumped by the Weyl constants W0 = 0x9E3779B9,
W1 = 0xBB67AE85 (mod 2^32).  Ten rounds are applied; the first round uses the
key as given.

The paper draws its delays from machine behaviour (Algorithm 1, Sec. 3.1.1);
the seeded Philox stream stands in for the network so that a delay map is a
pure function of (seed, step, PE, face).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0..c3) and key (k0, k1).

    Inputs are integers or integer arrays (broadcast together); outputs are
    uint32 arrays of the broadcast shape.
    """
    c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & MASK32
                              for v in (c0, c1, c2, c3, k0, k1))
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = (np.array(v, dtype=np.uint64) for v in (c0, c1, c2, c3))
    k0 = np.array(k0, dtype=np.uint64)
    k1 = np.array(k1, dtype=np.uint64)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0                     # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def split_seed(seed):
    """64-bit seed -> Philox key (k0 = low word, k1 = high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32
