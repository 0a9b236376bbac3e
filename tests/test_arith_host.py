"""CPU unit tests of the device arithmetic header (csrc/arith.cuh).

The header is compiled for the host with g++ (tests/host/arith_host_check.cpp)
and compared with exact Python integers: Montgomery multiplication and
set-up, modular doubling, Newton inverses, the multiply-by-inverse
divisibility test, and the strong tests.  The GPU kernels use the same
source; the GPU parity tests cover the kernels themselves.
"""
import ctypes
import math
import os
import random
import subprocess

import pytest

import numtheory as nt

HERE = os.path.dirname(os.path.abspath(__file__))
R = 1 << 64


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("arith") / "arith_host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so,
                    os.path.join(HERE, "host", "arith_host_check.cpp")], check=True)
    L = ctypes.CDLL(so)
    u64, u32, i32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
    for name, args, res in [("h_inv64", [u64], u64), ("h_inv32", [u32], u32),
                            ("h_mont_mul", [u64, u64, u64], u64), ("h_mod_dbl", [u64, u64], u64),
                            ("h_mont_setup", [u64, p], None), ("h_sprp2_64", [u64], i32),
                            ("h_sprp64", [u64, u64], i32), ("h_mont_mul32", [u32, u32, u32], u32),
                            ("h_sprp32", [u32, u32], i32), ("h_td64", [u64, i32], i32),
                            ("h_td32", [u32, i32], i32), ("h_td_prime", [i32], u32),
                            ("h_td2", [u64, i32], i32), ("h_td2_prime", [i32], u32),
                            ("h_td2_modulus", [i32], u32), ("h_td_pair", [u64], i32),
                            ("h_mont_residue32", [u64, u32], u32),
                            ("h_mont_mul_w", [u64, u64, u64], u64), ("h_mont_sqr_w", [u64, u64], u64),
                            ("h_mont_sqr_h", [u64, u64], u64),
                            ("h_mont_mul_f", [u64, u64, u64], u64), ("h_mont_sqr_f", [u64, u64], u64),
                            ("h_stress", [u64, u64, i32], u64),
                            ("h_jacobi", [ctypes.c_int64, u64], i32), ("h_is_square", [u64], i32),
                            ("h_jacobi_small", [ctypes.c_int32, u64], i32),
                            ("h_strong_lucas", [u64], i32)]:
        f = getattr(L, name)
        f.argtypes, f.restype = args, res
    return L


def _moduli(rng, k=300):
    ms = [3, 5, 2**32 + 15, 2**63 - 25, 2**63 + 1, 2**64 - 59, 2**64 - 1, (1 << 63) | 1]
    return ms + [rng.randrange(3, R) | 1 for _ in range(k)] + [rng.randrange(3, 2**40) | 1 for _ in range(50)]


def test_inverses(H):
    rng = random.Random(1)
    for n in _moduli(rng):
        assert (H.h_inv64(n) * n) % R == 1
        n32 = n & 0xFFFFFFFF | 1
        assert (H.h_inv32(n32) * n32) % (1 << 32) == 1


def test_mont_mul_and_setup(H):
    rng = random.Random(2)
    buf = (ctypes.c_uint64 * 6)()
    for n in _moduli(rng):
        rinv = pow(R, -1, n)
        for _ in range(10):
            a, b = rng.randrange(n), rng.randrange(n)
            assert H.h_mont_mul(a, b, n) == a * b * rinv % n
        for a, b in ((n - 1, n - 1), (0, n - 1), (n - 1, 1)):
            assert H.h_mont_mul(a, b, n) == a * b * rinv % n
        H.h_mont_setup(n, buf)
        q, one, mone, r2, ninv, r2w = list(buf)
        assert (q * n + 1) % (1 << 32) == 0 and ninv * n % R == 1 and r2w == r2
        assert one == R % n and mone == (n - R % n) and r2 == R * R % n


def test_word_level_montgomery(H):
    """Word-level REDC (wide multiply-adds) and the dedicated squaring."""
    rng = random.Random(12)
    for n in _moduli(rng, 1000):
        rinv = pow(R, -1, n)
        cases = [(n - 1, n - 1), (0, n - 1), (n - 1, 1), (0, 0), (1, 1), (n // 2, n - 2)]
        cases += [(rng.randrange(n), rng.randrange(n)) for _ in range(20)]
        for a, b in cases:
            assert H.h_mont_mul_w(a, b, n) == a * b * rinv % n, (a, b, n)
            assert H.h_mont_sqr_w(a, n) == a * a * rinv % n, (a, n)
            assert H.h_mont_sqr_h(a, n) == a * a * rinv % n, (a, n)
            assert H.h_mont_mul_f(a, b, n) == a * b * rinv % n, (a, b, n)
            assert H.h_mont_sqr_f(a, n) == a * a * rinv % n, (a, n)


@pytest.mark.parametrize("variant", range(6))
def test_montgomery_stress(H, variant):
    """2^20 random triples per formulation against 128-bit reference arithmetic."""
    assert H.h_stress(1234 + variant, 1 << 20, variant) == 0


def test_mod_dbl(H):
    rng = random.Random(3)
    for n in _moduli(rng):
        for x in [0, 1, n - 1, n // 2, (n + 1) // 2] + [rng.randrange(n) for _ in range(10)]:
            assert H.h_mod_dbl(x, n) == 2 * x % n


def test_strong_tests_against_python(H):
    rng = random.Random(4)
    vals = [rng.randrange(2**32, R) | 1 for _ in range(3000)]
    vals += [2**61 - 1, 2**63 - 25, 2**64 - 59, 3215031751, 2152302898747, 3474749660383]
    for n in vals:
        assert bool(H.h_sprp2_64(n)) == nt.strong_base2(n), n
        for a in (325, 9375, 1795265022):
            d, s = n - 1, 0
            while d % 2 == 0:
                d //= 2
                s += 1
            x = pow(a, d, n)
            ok = x in (1, n - 1) or any(pow(x, 1 << r, n) == n - 1 for r in range(1, s))
            assert bool(H.h_sprp64(n, a)) == ok, (n, a)


def test_sprp32_against_python(H):
    rng = random.Random(5)
    for n in [rng.randrange(3, 2**32) | 1 for _ in range(3000)] + [2047, 3277, 4033, 2**32 - 5]:
        for a in (2, 7, 61):
            if a % n == 0:
                continue
            d, s = n - 1, 0
            while d % 2 == 0:
                d //= 2
                s += 1
            x = pow(a, d, n)
            ok = x in (1, n - 1) or any(pow(x, 1 << r, n) == n - 1 for r in range(1, s))
            assert bool(H.h_sprp32(n, a % n)) == ok, (n, a)
        rinv = pow(1 << 32, -1, n)
        a, b = rng.randrange(n), rng.randrange(n)
        assert H.h_mont_mul32(a, b, n) == a * b * rinv % n


def test_divisibility_by_inverse(H):
    rng = random.Random(6)
    vals = [rng.randrange(R) for _ in range(2000)] + [0, 1, R - 1, 3 * 5 * 7 * 251]
    for i in range(53):
        p = H.h_td_prime(i)
        assert nt.trial_is_prime(p) and p % 2 == 1
        for v in vals + [p, p * (R // p - 1), p * rng.randrange(R // p)]:
            assert bool(H.h_td64(v, i)) == (v % p == 0)
            v32 = v & 0xFFFFFFFF
            assert bool(H.h_td32(v32, i)) == (v32 % p == 0)


def test_second_trial_stage(H):
    """td2_divisible (the base-2 kernel's second trial stage): its primes are
    the 72 odd primes after 53 in order, each group's modulus is the product
    of its three, and the Montgomery-reduced residue decides divisibility
    exactly as n % p does, on random values and on the edges of the
    reduction: n0 = 0 or 2^32 - 1, n1 = 2^32 - 1 (t close to 2^32 + m),
    multiples of each prime and of each modulus near 2^64, and m k + r for
    small r."""
    primes = [p for p in range(55, 500, 2) if nt.trial_is_prime(p)][:72]
    assert [H.h_td2_prime(i) for i in range(72)] == primes
    assert primes[0] == 59 and primes[-1] == 457
    for g in range(24):
        assert H.h_td2_modulus(g) == primes[3 * g] * primes[3 * g + 1] * primes[3 * g + 2] < 2**32
    rng = random.Random(27)
    vals = [rng.randrange(2**32, R) for _ in range(3000)]
    vals += [(rng.randrange(1, 2**32) << 32) for _ in range(200)]            # n0 = 0
    vals += [(rng.randrange(1, 2**32) << 32) | 0xFFFFFFFF for _ in range(200)]
    vals += [(0xFFFFFFFF << 32) | rng.randrange(2**32) for _ in range(300)]  # n1 = 2^32 - 1
    vals += [R - 1 - k for k in range(200)] + [2**32 + k for k in range(200)]
    for p in primes:
        vals += [p * (R // p - j) for j in range(3)] + [p * rng.randrange(2**32 // p, R // p)]
    for g in range(24):
        m = H.h_td2_modulus(g)
        vals += [m * (R // m - j) + r for j in range(2) for r in (0, 1, m - 1) if m * (R // m - j) + r < R]
        vals += [m * rng.randrange(1, R // m) + r for r in (0, 1, 2) for _ in range(3)]
    for groups in (1, 8, 12, 16, 24):
        ps = primes[:3 * groups]
        for v in vals:
            assert H.h_td2(v, groups) == int(any(v % p == 0 for p in ps)), (v, groups)
    assert H.h_td2(2**40, 5) == -1


def test_two_residue_trial_division(H):
    """td_pair_divisible (classify's td_fold 3): n is divisible by one of the
    odd primes 3..53 exactly when one of its two Montgomery residues (modulo
    29*31*41*43*47*53 and 3*5*7*11*13*17*19*23*37, both just below 2^32) is
    divisible by that prime; and mont_residue32 returns a value below 2^32
    congruent to n * 2^-32 modulo m, for moduli up to 2^32 - 1."""
    primes = [3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53]
    a, b = 29 * 31 * 41 * 43 * 47 * 53, 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23 * 37
    assert a == 3948078067 and b == 4127218095 and a * b == math.prod(primes)
    rng = random.Random(28)
    vals = [rng.randrange(2**32, R) for _ in range(4000)]
    vals += [(rng.randrange(1, 2**32) << 32) for _ in range(200)]
    vals += [(0xFFFFFFFF << 32) | rng.randrange(2**32) for _ in range(300)] + [R - 1 - k for k in range(300)]
    for m in (a, b) + tuple(primes):
        vals += [m * (R // m - j) + r for j in range(3) for r in (0, 1, m - 1) if m * (R // m - j) + r < R]
        vals += [m * rng.randrange(2**32 // m + 1, R // m) for _ in range(20)]
    for v in vals:
        assert H.h_td_pair(v) == int(any(v % p == 0 for p in primes)), v
    for m in (a, b, 3, 4294967291, 2**32 - 1, 65537):
        ri = pow(2**32, -1, m)
        for v in vals[:500] + [m, m * m % R, R - 1]:
            r = H.h_mont_residue32(v, m)
            assert r < 2**32 and r % m == v * ri % m, (v, m, r)


def test_jacobi_and_squares(H):
    rng = random.Random(21)
    for _ in range(3000):
        n = rng.randrange(3, R) | 1
        a = rng.randrange(-1000, 1000)
        assert H.h_jacobi(a, n) == nt.jacobi(a, n), (a, n)
        D = rng.choice([5, -7, 9, -11, 13, -15, 17, -19, 21, -23, 25, -27, 29, -31, 65535, -65535])
        assert H.h_jacobi_small(D, n) == nt.jacobi(D, n), (D, n)
    for _ in range(2000):
        r = rng.randrange(1, 1 << 32)
        assert H.h_is_square(r * r) == 1
        assert H.h_is_square(r * r - 1) == (r == 1)  # r^2 - 1 is a square only for r = 1
    assert H.h_is_square((1 << 64) - 1) == 0 and H.h_is_square(0) == 1


STRONG_LUCAS_PSEUDOPRIMES = [5459, 5777, 10877, 16109, 18971, 22499, 24569, 25199, 40309, 58519]


def test_strong_lucas_against_independent_python():
    """The independent Python test reproduces the known Selfridge strong Lucas
    pseudoprimes (OEIS A217255's first terms) and nothing else below 6*10^4."""
    found = [n for n in range(3, 60000, 2) if not nt.trial_is_prime(n)
             and int(math.isqrt(n)) ** 2 != n and nt.strong_lucas(n)]
    assert found == STRONG_LUCAS_PSEUDOPRIMES


def test_strong_lucas_device_source_on_large_values(H):
    rng = random.Random(22)
    vals = [rng.randrange(1 << 32, R) | 1 for _ in range(4000)]
    vals += [p for p in (2**61 - 1, 2**63 - 25, 2**64 - 59)]
    vals += [p * q for p, q in ((4294967291, 4294967279), (3037000493, 3037000453))]
    for n in vals:
        if any(n % p == 0 for p in (3, 5, 7, 11, 13)):
            continue
        if int(math.isqrt(n)) ** 2 == n:
            continue
        assert H.h_strong_lucas(n) == int(nt.strong_lucas(n)), n
    # squares are rejected
    assert H.h_strong_lucas(4294967291 ** 2) == 0
