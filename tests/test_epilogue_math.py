"""The integer identities the rank epilogue rests on (CPU, exact Python integers).

A term of Eq. 1's sum is floor(s 2^64 / d) for s <= d <= 65535 (s = S_ij, d = m_j).
The epilogue splits it as s Q + floor(s r / d), Q = floor((2^64 - 1) / d),
r = 2^64 - Q d in [1, d], and takes the small floor as one fixed-point product
floor(s W / 2^63) with W = ceil(2^63 r / d), computed by two steps of long division.
"""
import random


M64 = (1 << 64) - 1


def floor_weight(d):
    q = M64 // d
    r = (1 << 64) - q * d
    n1 = r << 47
    q1, r1 = divmod(n1, d)
    n2 = r1 << 16
    q2, r2 = divmod(n2, d)
    return q, r, (q1 << 16) + q2 + (1 if r2 else 0)


def small_floor(s, w):
    # the device's form: hi32(s Whi + umulhi(s, Wlo)) of the 64-bit sum, shifted by 31
    wlo, whi = w & 0xFFFFFFFF, w >> 32
    return (s * whi + ((s * wlo) >> 32)) >> 31


def test_split_and_weight_for_every_divisor():
    rng = random.Random(7)
    for d in range(1, 65536):
        q, r, w = floor_weight(d)
        assert 1 <= r <= d and w <= 1 << 63
        assert w == -((-(r << 63)) // d)  # the long division gives the ceiling
        for s in (0, 1, d - 1, d, rng.randrange(0, d + 1)):
            assert small_floor(s, w) == (s * r) // d
            assert s * q + small_floor(s, w) == (s << 64) // d


def test_every_shared_count_on_some_divisors():
    for d in (1, 2, 3, 7, 255, 256, 300, 4097, 65521, 65535):
        q, r, w = floor_weight(d)
        for s in range(0, d + 1):
            assert small_floor(s, w) == (s * r) // d


def test_row_and_column_sums_fit_their_words():
    """A tile adds at most 128 terms (each <= 2^64) per row or column: T < 2^72, so
    T >> 32 < 2^40, and fewer than 2^17 adds per key keep both 64-bit words of the
    key accumulator (T mod 2^32 and T >> 32) below 2^57."""
    t_max = 128 * (1 << 64)
    assert t_max < 1 << 72 and (t_max >> 32) < 1 << 40
    assert (1 << 17) * (1 << 40) <= 1 << 57 and (1 << 17) * (1 << 32) < 1 << 64
    # the row's partial sums over 64 columns: s Qlo and s Qhi each below 2^54
    assert 64 * 65535 * M64 >> 32 < 1 << 54
