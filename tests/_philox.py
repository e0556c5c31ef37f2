"""Philox-4x32-10 written from its published definition (Salmon, Moraes, Dror
and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds
of two 32x32->64-bit multiplications by 0xD2511F53 and 0xCD9E8D57 with a
Weyl key schedule (0x9E3779B9, 0xBB67AE85).  Test-side reference only."""

MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    c = [x & MASK for x in counter]
    k = [x & MASK for x in key]
    for _ in range(10):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [(p1 >> 32) ^ c[1] ^ k[0], p1 & MASK, (p0 >> 32) ^ c[3] ^ k[1], p0 & MASK]
        k = [(k[0] + 0x9E3779B9) & MASK, (k[1] + 0xBB67AE85) & MASK]
    return c
