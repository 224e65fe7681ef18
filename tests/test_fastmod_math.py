"""The device computes r = h mod (n-1) without a 64-bit divide, by the direct
remainder of Lemire, Kaser & Kurz (2019): with c = ceil(2^96 / D),
h mod D = ((c * h mod 2^96) * D) >> 96 for every h < 2^64 when D < 2^31.
This checks that identity (and the limb split the kernel uses) in exact
integer arithmetic on random and extreme values; the CUDA code itself is
checked against the oracle's partner draws on the GPU."""
import random

M64 = (1 << 64) - 1
M32 = (1 << 32) - 1


def direct_mod(h: int, D: int) -> int:
    if D == 1:
        return 0
    c = -(-(1 << 96) // D)
    c_lo, c_hi = c & M64, c >> 64
    assert c_hi < (1 << 32)
    l_lo = (c_lo * h) & M64
    p_hi = (c_lo * h) >> 64
    l_hi = ((p_hi & M32) + c_hi * (h & M32)) & M32
    acc = l_hi * D + ((l_lo * D) >> 64)
    assert acc < (1 << 64)
    return acc >> 32


def test_direct_remainder_identity():
    rng = random.Random(0)
    divisors = [1, 2, 3, 5, 7, 1000, 999_999, 123_456_789, 2**31 - 2, 2**31 - 3, 2**30,
                2**30 + 1, 65_535, 65_537] + [rng.randrange(1, 2**31 - 1) for _ in range(300)]
    for D in divisors:
        values = [0, 1, D - 1, D, D + 1, M64, M64 - 1, (M64 // D) * D, (M64 // D) * D - 1,
                  1 << 63, (1 << 32) - 1, 1 << 32] + [rng.getrandbits(64) for _ in range(300)]
        for h in values:
            h &= M64
            assert direct_mod(h, D) == h % D, (h, D)
