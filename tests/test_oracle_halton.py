"""Pins for the oracle's QMC sampling (Appendix A.2): exact radical inverse,
digit scrambling, full-screen sample enumeration."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def phi_fraction(b, f, i):
    """Radical inverse written with Python rationals (independent of C)."""
    acc, scale = Fraction(0), Fraction(1, b)
    while i > 0:
        d = i % b
        i //= b
        acc += ((f * d) % b) * scale
        scale /= b
    return acc


def test_primes():
    assert [oracle.prime(d) for d in range(10)] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    assert oracle.prime(113) == 619  # 2 + 7 * 16 dimensions end at the 114th prime


def test_radical_inverse_matches_rationals():
    rng = np.random.default_rng(1)
    cases = [(2, 1), (3, 1), (5, 3), (7, 4), (619, 400), (113, 57)]
    idx = [0, 1, 2, 3, 17, 2**24 - 1, 2**32 - 1, 2**32, 2**53 + 7, 2**63 - 25, 2**64 - 1]
    idx += [int(x) for x in rng.integers(0, 2**63, 200, dtype=np.int64)]
    for b, f in cases:
        for i in idx:
            want = int(phi_fraction(b, f, i) * 2**32)  # floor of a positive rational
            assert oracle.radical_inverse_u32(b, f, i) == want, (b, f, i)


def test_base2_is_bit_reversal():
    rng = np.random.default_rng(2)
    for i in [int(x) for x in rng.integers(0, 2**63, 500, dtype=np.int64)] + [2**64 - 1, 1, 2]:
        low = i & 0xFFFFFFFF
        rev = int(f"{low:032b}"[::-1], 2)
        assert oracle.radical_inverse_u32(2, 1, i) == rev


@pytest.mark.parametrize("b", [3, 5, 7, 11, 13])
def test_scramble_is_a_digit_bijection_fixing_zero(b):
    for seed in (0, 1, 17050126):
        f = oracle.scramble_factor(seed, b)
        assert 2 <= f < b
        assert sorted((f * d) % b for d in range(b)) == list(range(b))
    assert oracle.scramble_factor(5, 2) == 1


@pytest.mark.parametrize("b,m", [(2, 10), (3, 6), (5, 4), (7, 3), (13, 2)])
def test_elementary_intervals_one_point_each(b, m):
    f = oracle.scramble_factor(123, b)
    n = b**m
    for block in (0, 1, 977):
        ids = range(block * n, (block + 1) * n)
        cells = [int(phi_fraction(b, f, i) * n) for i in ids]
        assert sorted(cells) == list(range(n))
        # the oracle's fixed-point values sit in the same cells (floor of the
        # exact value, so a point on a cell boundary stays in its cell)
        got = [((oracle.radical_inverse_u32(b, f, i) + 1) * n - 1) >> 32 for i in ids]
        assert got == cells


@pytest.mark.parametrize("W,H", [(1, 1), (7, 5), (64, 64), (33, 10)])
def test_pixel_enumeration_lands_in_pixel(W, H):
    k = max(0, (W - 1).bit_length())
    l = 0
    while 3**l < H:
        l += 1
    P = 2**k * 3**l
    seen = set()
    for y in range(H):
        for x in range(W):
            i0 = oracle.pixel_base_index(W, H, x, y)
            assert 0 <= i0 < P and i0 not in seen
            seen.add(i0)
            for j in (0, 1, 5, 1000003):
                i = i0 + j * P
                assert int(phi_fraction(2, 1, i) * 2**k) == x
                assert int(phi_fraction(3, 1, i) * 3**l) == y


def test_sample_dims_batch_definition():
    W, H, seed = 64, 64, 99
    idx = np.array([0, 5, 2**40 + 3, 2**63 + 11], np.uint64)
    u = oracle.sample_dims_u32(idx, 12, W, H, seed)
    for r, i in enumerate(idx.tolist()):
        assert u[r, 0] == int(phi_fraction(2, 1, i >> 6) * 2**32)   # 2^6 = 64 >= W
        assert u[r, 1] == int(phi_fraction(3, 1, i // 81) * 2**32)  # 3^4 = 81 >= H
        for d in range(2, 12):
            b = oracle.prime(d)
            assert u[r, d] == int(phi_fraction(b, oracle.scramble_factor(seed, b), i) * 2**32)
