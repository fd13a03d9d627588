"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
published round function: two 64x64->128 multiplies per round with the
multipliers 0xD2E7470EE14C6C93 / 0xCA5A826395121157 and the Weyl key bumps
0x9E3779B97F4A7C15 / 0xBB67AE8584CAA73B, 10 rounds.

Pinned: against numpy.random.Philox (an independent implementation of the
same published generator) in tests/test_oracle_philox.py.

Stream layout used by the sampler (both sides implement it): counter
(sweep, link, 0, 0), key (seed, chain); output word 0 -> acceptance uniform,
word 1 -> proposal uniform; uniform = (word >> 11) * 2^-53 in [0, 1).
"""
M64 = (1 << 64) - 1
_M0, _M1 = 0xD2E7470EE14C6C93, 0xCA5A826395121157
_W0, _W1 = 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B


def philox4x64_10(ctr, key):
    c0, c1, c2, c3 = (int(x) & M64 for x in ctr)
    k0, k1 = (int(x) & M64 for x in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 64, p0 & M64
        hi1, lo1 = p1 >> 64, p1 & M64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0, k1 = (k0 + _W0) & M64, (k1 + _W1) & M64
    return c0, c1, c2, c3


def uniform53(word: int) -> float:
    return (int(word) >> 11) * (1.0 / 9007199254740992.0)


def draws(seed: int, chain: int, sweep: int, link: int):
    """(u_accept, u_propose) for one proposal."""
    w = philox4x64_10((sweep, link, 0, 0), (seed, chain))
    return uniform53(w[0]), uniform53(w[1])


def draws4(seed: int, chain: int, sweep: int, link: int):
    """All four words of one proposal's block as uniforms (u_accept,
    u_propose, u_axis_z, u_axis_phi); the last two serve SU(2) proposals."""
    w = philox4x64_10((sweep, link, 0, 0), (seed, chain))
    return tuple(uniform53(x) for x in w)
