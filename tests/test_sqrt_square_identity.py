"""Exhaustive check of the identity the kernels use for lambda = 1, C = 1.

With lambda = 1 the spatial term is (1 - 1) * s2 = +0 and the edge cost is
sqrt_rn(+0 + 1 * fl(d * d)) = sqrt_rn(fl(d * d)).  In IEEE binary32 with
round-to-nearest this equals |d| whenever d * d neither underflows to the
subnormal range nor overflows; the kernels use |d| for 2^-63 <= |d| <= 2^63
and d = 0, and the square root otherwise.  This test checks the identity for
every float32 value in that range (about 1.06e9 values, both signs follow from
the square), so the shortcut is exact, not an approximation.
"""
import numpy as np

LO = 0x20000000  # 2^-63
HI = 0x5F000000  # 2^63


def test_sqrt_of_square_is_abs_on_the_whole_range():
    chunk = 1 << 24
    bad = 0
    for start in range(LO, HI + 1, chunk):
        stop = min(start + chunk, HI + 1)
        d = np.arange(start, stop, dtype=np.uint32).view(np.float32)
        sq = d * d
        r = np.sqrt(sq)
        bad += int(np.count_nonzero(r != d))
    assert bad == 0
    # the range ends are what the kernels test against
    assert np.float32(2.0**-63).view(np.uint32) == LO
    assert np.float32(2.0**63).view(np.uint32) == HI


def test_identity_fails_just_outside_the_range():
    """Below 2^-63 the square is subnormal and the identity breaks for some
    values, which is why the kernels fall back to the square root there."""
    d = np.arange(0x1F000000, LO, 4099, dtype=np.uint32).view(np.float32)
    assert np.any(np.sqrt(d * d) != d)
    big = np.float32(3.5e19)
    assert np.isinf(big * big)
