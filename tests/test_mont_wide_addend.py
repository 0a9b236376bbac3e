"""Word-level algebra of Montgomery formulations 7 and 8 (CPU model).

The device code forms a b R^-1 mod n (R = 2^64) in 32-bit words with wide
products that take a 64-bit addend (PTX mad.wide.u32), so that partial sums
need no separate carry chains:

  U  = a0 b1 + hi(a0 b0)             V  = a1 b0 + lo(U)
  T  = a1 b1 + hi(U) + hi(V)         a b = T 2^64 + lo(V) 2^32 + lo(a0 b0)
  m  = lo64(a b) n^-1 mod 2^64
  V2 = m1 n0 + lo(m0 n1)             W2 = m1 n1 + hi(m0 n1) + hi(V2)
  hi64(m n) = W2 + c,  c = [lo(V2) > bits 32..63 of a b]
  r  = T - W2 - c, plus n when negative.

Every sum above stays below 2^64, and m0 n0 is never formed (its low word
equals that of a b).  This test replays those word operations with exact
integers and checks r against a b R^-1 mod n, and each no-overflow claim,
on adversarial and random odd moduli.  It imports no library code.
"""
import random

import pytest

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def _wide(x, y, addend=0):
    v = x * y + addend
    assert v <= M64  # the claim: the 64-bit addend never overflows the product
    return v


def _mont_words(a, b, n, ninv, square_three_products=False):
    a0, a1, b0, b1 = a & M32, a >> 32, b & M32, b >> 32
    n0, n1, i0, i1 = n & M32, n >> 32, ninv & M32, ninv >> 32
    p00 = a0 * b0
    t0, h = p00 & M32, p00 >> 32
    if square_three_products:
        assert a == b
        c = a0 * a1
        u = c + h
        v = c + (u & M32)
        assert u <= M64 and v <= M64
    else:
        u = _wide(a0, b1, h)
        v = _wide(a1, b0, u & M32)
    t1 = v & M32
    T = _wide(a1, b1, (u >> 32) + (v >> 32))
    assert T * 2**64 + t1 * 2**32 + t0 == a * b
    m0 = (t0 * i0) & M32
    m1 = ((t0 * i0 >> 32) + t0 * i1 + t1 * i0) & M32
    m = m0 | (m1 << 32)
    assert m == ((t0 | (t1 << 32)) * ninv) & M64
    q01 = m0 * n1
    v2 = _wide(m1, n0, q01 & M32)
    w2 = _wide(m1, n1, (q01 >> 32) + (v2 >> 32))
    c = 1 if (v2 & M32) > t1 else 0
    assert w2 + c == (m * n) >> 64
    r = T - w2 - c
    assert -n < r < n
    return r + n if r < 0 else r


def _moduli(rng):
    fixed = [2**32 + 15, 2**33 - 9, 2**63 - 25, 2**63 + 29, 2**64 - 59, 2**64 - 1,
             (1 << 64) - (1 << 32) + 1, 0xFFFFFFFF00000001 | 1, 3, 2**40 + 1]
    return fixed + [rng.getrandbits(b) | (1 << (b - 1)) | 1 for b in range(2, 65) for _ in range(3)]


@pytest.mark.parametrize("square", [False, True])
def test_wide_addend_montgomery_matches_definition(square):
    rng = random.Random(77 + square)
    for n in _moduli(rng):
        if n < 3:
            continue
        ninv = pow(n, -1, 1 << 64)
        rinv = pow(1 << 64, -1, n)
        xs = {0, 1, n - 1, n - 2, n // 2}
        xs.update(rng.randrange(n) for _ in range(6))
        for a in xs:
            for b in ([a] if square else xs):
                got = _mont_words(a, b, n, ninv, square_three_products=square)
                assert got == a * b * rinv % n, (a, b, n)
