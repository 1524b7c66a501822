"""The e4m3 kernels' epilogue reduces y mod p by an invariant-divisor multiply: floor(y / p) =
floor(y * mp / 2^32) with mp = ceil(2^32 / p) = (2^32 + e) / p, 0 <= e < p.  The product exceeds
y / p by y e / (p 2^32) < y / 2^32, and the fractional part of y / p is at most 1 - 1/p, so the
floor is exact whenever y < 2^32 / p: for every y < 2^23 when p < 2^9 and every y < 2^24 when
p < 2^8.  Checked here exhaustively on the ranges the kernels use (sums below 2^23 for the
primes of the pre-tiled route, below 2^24 for those of the TMA route), and shown to fail far
past the bound, so the check has teeth."""
import numpy as np
import pytest


def mulhi_mod(y, p):
    mp = np.uint64((0xFFFFFFFF // p) + 1)          # ceil(2^32 / p) for p >= 2
    q = (y * mp) >> np.uint64(32)
    return y - np.uint64(p) * q


@pytest.mark.parametrize("p", [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 127, 251, 509])
def test_exact_below_2_23(p):
    y = np.arange(1 << 23, dtype=np.uint64)
    assert np.array_equal(mulhi_mod(y, p), y % np.uint64(p))


@pytest.mark.parametrize("p", [2, 3, 5, 7, 11, 13, 17])
def test_exact_below_2_24_small_p(p):
    y = np.arange(1 << 24, dtype=np.uint64)
    assert np.array_equal(mulhi_mod(y, p), y % np.uint64(p))


def test_fails_past_the_bound():
    # a large p and y far past 2^23: the error term reaches 1 / p and some residue comes out wrong
    p = 65521
    y = np.arange(1 << 31, (1 << 31) + (1 << 22), dtype=np.uint64)
    assert not np.array_equal(mulhi_mod(y, p), y % np.uint64(p))
