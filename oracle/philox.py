"""Philox4x32-10 counter-based generator (test infrastructure; see package header).

Written from its published definition (J. K. Salmon, M. A. Moraes, R. O. Dror,
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit
counter and a 2 x 32-bit key; each of 10 rounds multiplies words 0 and 2 by
fixed odd constants, and recombines the high/low halves with the other two
words and the round key; the key is bumped by Weyl constants between rounds.

The paper itself names no generator; the counter layout below is the reading
this project uses on both sides (CPU oracle and CUDA kernels implement it
separately):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (site, slice - 1, 2*sweep + pass, chain | domain << 24)
with domain 0 for Metropolis proposals and 1 for the initial field, and
pass 0 (up) / 1 (down). One draw per proposal, used or not.
"""

import numpy as np

MUL0 = 0xD2511F53
MUL1 = 0xCD9E8D57
WEYL0 = 0x9E3779B9
WEYL1 = 0xBB67AE85
_M32 = np.uint64(0xFFFFFFFF)

DOMAIN_METROPOLIS = 0
DOMAIN_INIT = 1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. Counters are broadcastable integer arrays
    (taken mod 2^32), the key two integers. Returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _M32 for c in (c0, c1, c2, c3))
    k0 = np.uint64(k0 & 0xFFFFFFFF)
    k1 = np.uint64(k1 & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(WEYL0)) & _M32
            k1 = (k1 + np.uint64(WEYL1)) & _M32
        p0 = np.uint64(MUL0) * c0
        p1 = np.uint64(MUL1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def key_of(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def uniform53(r0, r1):
    """u in [0, 1) with 53 random bits: ((r0 >> 5) * 2^26 + (r1 >> 6)) * 2^-53."""
    hi = (np.asarray(r0, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    lo = (np.asarray(r1, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0)


def metropolis_uniforms(seed, chain, sweep, pas, slice1, n_sites):
    """The uniforms for all proposals of one slice visit (slice1 is 1-based)."""
    k0, k1 = key_of(seed)
    site = np.arange(n_sites, dtype=np.uint64)
    r = philox4x32_10(site, slice1 - 1, 2 * sweep + pas,
                      (chain & 0xFFFFFF) | (DOMAIN_METROPOLIS << 24), k0, k1)
    return uniform53(r[0], r[1])


def initial_field(seed, chain, n_slices, n_sites):
    """Initial Ising field s[l-1, i] = +1 if the low bit of word 0 is set, else -1."""
    k0, k1 = key_of(seed)
    site = np.arange(n_sites, dtype=np.uint64)[None, :]
    sl = np.arange(n_slices, dtype=np.uint64)[:, None]
    r = philox4x32_10(site, sl, 0, (chain & 0xFFFFFF) | (DOMAIN_INIT << 24), k0, k1)
    return np.where((r[0] & np.uint32(1)) == 1, 1, -1).astype(np.int8)
