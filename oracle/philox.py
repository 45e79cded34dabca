"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written from its published definition.

The paper's own generator (SFMT, Sec. 3.1.1) is replaced by this
counter-based one so that every (walker, proposal) draw is reproducible on
any device.  Pure Python integers; slow by design.
"""
MASK32 = 0xFFFFFFFF
# Round multipliers and key-schedule (Weyl) increments from the SC'11 paper.
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(ctr, key):
    """Return the 4 output words for counter ctr (4 words) and key (2 words)."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for _ in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
        k0 = (k0 + PHILOX_W0) & MASK32
        k1 = (k1 + PHILOX_W1) & MASK32
    return c0, c1, c2, c3


def mulhi(r: int, n: int) -> int:
    """floor(r * n / 2^32): maps a 32-bit word to 0..n-1."""
    return (int(r) * int(n)) >> 32


def uniform24(r: int) -> float:
    """(r >> 8) * 2^-24: a uniform in [0, 1) exact in FP32 and FP64."""
    return float(int(r) >> 8) * (1.0 / 16777216.0)


def proposal_draw(seed: int, system: int, walker: int, counter: int):
    """The four words of proposal `counter` of a walker: counter block
    (counter_lo, counter_hi, walker, system), key (seed_lo, seed_hi)."""
    return philox4x32_10(
        (counter & MASK32, (counter >> 32) & MASK32, walker, system),
        (seed & MASK32, (seed >> 32) & MASK32))


def exchange_threshold(p_exchange: float) -> int:
    """An exchange is proposed iff r0 < threshold (threshold up to 2^32)."""
    return min(int(p_exchange * 4294967296.0), 4294967296)
