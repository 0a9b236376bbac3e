"""The quotient estimate behind the base-2 kernel's "multiply by 2^w".

For odd n >= 2^32, x < n and 0 <= w <= 15 the kernel forms x 2^w mod n as
x 2^w - q n, with q estimated in single precision from the top 32 bits of x
and n after normalising n (clz), one reciprocal, one product and one fused
multiply-add that also subtracts 1/32.  Its correctness rests on the estimate
being floor(x 2^w / n) or one less (the remainder is then in [0, 2n) and one
conditional subtraction finishes it).  This test emulates each IEEE single
operation with exact rational arithmetic and correct rounding, and checks that
claim on adversarial and random inputs.  The integer form of the estimate
(base2_window 2: a 32-bit reciprocal rcp = min(floor(inv 2^63), 2^32 - 1) from
the same single-precision inv, e = floor(xt rcp / 2^32), q = max(e - 2^10, 0)
>> (31 - w)) is checked the same way.  CPU only; it imports no library code.
"""
from fractions import Fraction
import random

import numpy as np
import pytest


def _round_f32(v: Fraction) -> Fraction:
    """v rounded to the nearest IEEE single (ties to even); normal range only."""
    if v == 0:
        return Fraction(0)
    sign = -1 if v < 0 else 1
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scaled = a * Fraction(2) ** (23 - e)  # in [2^23, 2^24)
    lo = scaled.numerator // scaled.denominator
    rem = scaled - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return sign * Fraction(lo) * Fraction(2) ** (e - 23)


def _estimate(x: int, w: int, n: int) -> int:
    sh = 64 - n.bit_length()
    nt = ((n << sh) >> 32) & 0xFFFFFFFF
    xt = ((x << sh) >> 32) & 0xFFFFFFFF
    inv = _round_f32(1 / _round_f32(Fraction(nt)))
    m = _round_f32(_round_f32(Fraction(xt)) * inv)
    v = _round_f32(m * 2 ** w - Fraction(1, 32))  # one rounding: the FMA
    v = max(v, Fraction(0))
    return v.numerator // v.denominator  # truncation = floor for v >= 0


def test_rounding_helper_matches_numpy():
    rng = np.random.default_rng(7)
    for a in rng.integers(1, 2**32, size=200, dtype=np.uint64):
        assert _round_f32(Fraction(int(a))) == Fraction(float(np.float32(a)))
    for a in rng.integers(2**31, 2**32, size=100, dtype=np.uint64):
        want = np.float32(1) / np.float32(a)
        assert _round_f32(1 / _round_f32(Fraction(int(a)))) == Fraction(float(want))


def _moduli(rng):
    fixed = [2**32 + 1, 2**32 + 15, 2**33 - 9, 2**40 + 15, 2**48 + 21, 2**63 - 25, 2**63 + 29,
             2**63 + 1, 2**64 - 59, 2**64 - 1, 3 * 2**62 + 1, 2**62 + 1]
    rand = [rng.getrandbits(b) | (1 << (b - 1)) | 1 for b in range(33, 65) for _ in range(2)]
    return fixed + rand


@pytest.mark.parametrize("w", range(16))
def test_estimate_is_q_or_q_minus_one(w):
    rng = random.Random(1000 + w)
    for n in _moduli(rng):
        xs = {0, 1, n - 1, n - 2, n // 2, (n + 1) // 2}
        xs.update(rng.randrange(n) for _ in range(4))
        for _ in range(4):  # x 2^w / n just above and just below an integer k
            k = rng.randrange(1, 2**w + 1)
            lo = (k * n) >> w
            xs.update(v for v in (lo - 1, lo, lo + 1) if 0 <= v < n)
        for x in xs:
            q = (x << w) // n
            est = _estimate(x, w, n)
            assert est in (q, q - 1), (x, w, n, q, est)
            r = (x << w) - est * n
            assert 0 <= r < 2 * n


def _estimate_int(x: int, w: int, n: int) -> int:
    sh = 64 - n.bit_length()
    nt = ((n << sh) >> 32) & 0xFFFFFFFF
    xt = ((x << sh) >> 32) & 0xFFFFFFFF
    inv = _round_f32(1 / _round_f32(Fraction(nt)))
    scaled = _round_f32(inv * 2**63)  # exact: a power-of-two scaling
    rcp = min(scaled.numerator // scaled.denominator, 2**32 - 1)
    e = (xt * rcp) >> 32
    return max(e - 1024, 0) >> (31 - w)


@pytest.mark.parametrize("w", range(16))
def test_integer_estimate_is_q_or_q_minus_one(w):
    rng = random.Random(2000 + w)
    moduli = _moduli(rng) + [(1 << 63) | 1, (1 << 63) + 2**32 + 1, 2**32 + 2**31 + 1,
                             (2**32 - 1) << 32 | 1]  # top words at 2^31 (rcp saturates) and 2^32 - 1
    for n in moduli:
        xs = {0, 1, n - 1, n - 2, n // 2, (n + 1) // 2}
        xs.update(rng.randrange(n) for _ in range(4))
        for _ in range(6):  # x 2^w / n just above and just below an integer k
            k = rng.randrange(1, 2**w + 1)
            lo = (k * n) >> w
            xs.update(v for v in (lo - 1, lo, lo + 1) if 0 <= v < n)
        for x in xs:
            q = (x << w) // n
            est = _estimate_int(x, w, n)
            assert est in (q, q - 1), (x, w, n, q, est)


def test_integer_estimate_needs_its_bias():
    """Without the bias of 2^10 the integer estimate overshoots floor(x 2^w / n)
    for some inputs (x 2^w / n just below an integer), so the bias is needed."""
    rng = random.Random(99)
    over = 0
    for n in _moduli(rng):
        sh = 64 - n.bit_length()
        nt = ((n << sh) >> 32) & 0xFFFFFFFF
        inv = _round_f32(1 / _round_f32(Fraction(nt)))
        scaled = _round_f32(inv * 2**63)
        rcp = min(scaled.numerator // scaled.denominator, 2**32 - 1)
        for w in (0, 7, 15):
            for k in range(1, 40):
                x = ((k * n) >> w)  # x 2^w / n just below k
                if x >= n:
                    continue
                xt = ((x << sh) >> 32) & 0xFFFFFFFF
                if ((xt * rcp) >> 32) >> (31 - w) > (x << w) // n:
                    over += 1
    assert over > 0
