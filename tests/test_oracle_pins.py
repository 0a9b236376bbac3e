"""Pins of the CPU oracle against the paper and against mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden, with their section), closed forms, brute force
by independent code (tests/numtheory.py), Lucas/Pratt certificates, and
invariants (Carmichael numbers, strong pseudoprimes).  CPU only.
"""
import math
import os
import random

import numpy as np
import pytest

import oracle
import numtheory as nt
from workloads import plain_small, plain_large, bitlen_uniform, load_pool

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_kv(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = [int(x) for x in v.split()]
    return out


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- paper values

def test_sec1_worked_example():
    g = _read_kv("sec1_example.txt")
    out = oracle.isprime_u64(np.array(g["input"], dtype=np.uint64))
    assert out.tolist() == g["output"]


def test_table1_division_counts():
    """Sec. 6, Table 1: the oracle's sieve reproduces every printed count."""
    for n_str, count_str in _read_rows("table1_division_counts.txt"):
        N, expect = int(n_str), int(count_str)
        assert oracle.division_count(N) == expect, N
        # closed form of the same double sum: sum over primes p <= sqrt(N) of (N - p)
        ps = oracle.primes_upto(math.isqrt(N)).astype(object)
        assert sum(N - int(p) for p in ps) == expect


def test_eq5_eq6_wheel():
    g = _read_kv("eq5_wheel_2357.txt")
    cyc = oracle.wheel_diffs()
    assert cyc == g["cycle"]
    assert sum(cyc) == 210 and len(cyc) == 48
    assert (1 + np.cumsum(cyc[:6])).tolist() == g["first_six"]
    assert oracle.wheel_diffs_mod(6) == g["wheel_23"]
    assert oracle.wheel_diffs_mod(30) == g["wheel_235"]


def test_sec6_shrink_percentages():
    """Sec. 6.1.2: the fraction removed by the first primes, truncated."""
    for primes, pct in _read_rows("sec6_shrink_percent.txt"):
        P = math.prod(int(p) for p in primes.split(","))
        kept = len(oracle.wheel_diffs_mod(P)) if P > 2 else 1
        removed = 100.0 * (1 - kept / P)
        assert int(removed) == int(pct), (primes, removed)


# ---------------------------------------------------------------- arithmetic

def test_modadd_and_mulmods_against_python_ints():
    rng = random.Random(7)
    mods = [3, 5, 2**32 - 5, 2**32 + 15, 2**63 - 25, 2**63 + 1, 2**64 - 59, 2**64 - 1]
    mods += [rng.randrange(3, 2**64) | 1 for _ in range(200)]
    for m in mods:
        for _ in range(20):
            a, b = rng.randrange(m), rng.randrange(m)
            assert oracle.modadd(a, b, m) == (a + b) % m
            assert oracle.mulmod(a, b, m) == a * b % m
            assert oracle.mulmod_classic(a, b, m) == a * b % m
        for a, b in ((m - 1, m - 1), (m - 1, 1), (0, m - 1), (m - 2, m - 1)):
            assert oracle.mulmod(a, b, m) == a * b % m
            assert oracle.mulmod_classic(a, b, m) == a * b % m
            assert oracle.modadd(a, b, m) == (a + b) % m


def test_powmod_against_python_pow():
    rng = random.Random(11)
    for _ in range(500):
        m = rng.randrange(2, 2**64)
        a = rng.randrange(2**64)
        e = rng.randrange(2**64)
        assert oracle.powmod(a, e, m) == pow(a, e, m)
    assert oracle.powmod(5, 0, 7) == 1
    assert oracle.powmod(5, 0, 1) == 0


def test_sprp_matches_independent_base2_test():
    rng = random.Random(3)
    vals = [rng.randrange(3, 2**64) | 1 for _ in range(3000)]
    vals += [2047, 3277, 4033, 4681, 8321]  # base-2 strong pseudoprimes
    vals += list(range(3, 200_000, 2))       # every small odd n, prime or not
    for n in vals:
        assert oracle.sprp(n, 2) == nt.strong_base2(n), n


# ---------------------------------------------------------------- brute force

def test_trial_branch_against_sieve_below_1e6():
    N = 10**6
    ref = nt.simple_sieve(N - 1)
    out = oracle.isprime_u64(np.arange(N, dtype=np.uint64))
    assert np.array_equal(out.astype(bool), ref)
    assert int(out.sum()) == 78498  # pi(10^6)


def test_pi_1e8():
    assert oracle.count_primes(0, 10**8) == 5761455


@pytest.mark.slow
def test_pi_1e9():
    """pi(10^9) = 50,847,534, counted with the oracle's classifier."""
    assert oracle.count_primes(0, 10**9) == 50847534


def test_mr_branch_against_segmented_sieve_at_2p24():
    lo, hi = 1 << 24, (1 << 24) + (1 << 22)
    ref = nt.window_sieve(lo, hi)
    out = oracle.isprime_u64(np.arange(lo, hi, dtype=np.uint64))
    assert np.array_equal(out.astype(bool), ref)


def test_mr_branch_against_segmented_sieve_at_2p32():
    lo, hi = 1 << 32, (1 << 32) + (1 << 23)
    ref = nt.window_sieve(lo, hi)
    out = oracle.isprime_u64(np.arange(lo, hi, dtype=np.uint64))
    assert np.array_equal(out.astype(bool), ref)


def test_mr_branch_at_2p50_window():
    """Window near 2^50: sieve by all primes below 2^25."""
    lo, hi = (1 << 50) - (1 << 20), (1 << 50) + (1 << 20)
    ref = nt.window_sieve(lo, hi)
    out = oracle.isprime_u64(np.arange(lo, hi, dtype=np.uint64))
    assert np.array_equal(out.astype(bool), ref)


def test_top_of_range_by_factoring_and_certificates():
    """The last 2^12 integers below 2^64: composites are factored by
    Pollard-Brent, primes get a Lucas (Pratt) certificate."""
    lo = (1 << 64) - (1 << 12)
    vals = np.arange(lo, 1 << 64, dtype=np.uint64)
    out = oracle.isprime_u64(vals)
    rng = random.Random(99)
    for v, f in zip(vals.tolist(), out.tolist()):
        if f:
            assert nt.pratt_prime(v, rng), v
        else:
            fac = nt.factorize(v, rng)
            assert sum(fac.values()) >= 2 and math.prod(p**e for p, e in fac.items()) == v


def test_wheel_method_agrees_on_medium_integers():
    """Sec. 3's wheel trial division is an independent algorithm."""
    vals = bitlen_uniform(5, 3000, 2, 40)
    out = oracle.isprime_u64(vals)
    for v, f in zip(vals.tolist(), out.tolist()):
        assert oracle.isprime_wheel(v) == bool(f), v


# ---------------------------------------------------------------- special cases

KNOWN_PRIMES = [2, 3, 5, 2**31 - 1, 2**32 - 5, 2**32 + 15, 2**48 - 59, 2**52 - 47,
                2**53 - 111, 2**61 - 1, 2**62 - 57, 2**63 - 25, 2**64 - 59]


def test_known_primes_have_certificates_and_pass():
    rng = random.Random(1)
    for p in KNOWN_PRIMES:
        assert nt.pratt_prime(p, rng), p
        assert oracle.isprime1(p), p


def test_special_composites_and_small_values():
    assert [oracle.isprime1(v) for v in range(6)] == [False, False, True, True, False, True]
    assert not oracle.isprime1(2**64 - 1)       # divisible by 3
    assert not oracle.isprime1(2**32 + 1)       # 641 * 6700417
    assert not oracle.isprime1(2**32 - 1)
    for v in range(2**64 - 57, 2**64, 2):       # no prime above 2^64 - 59
        assert not oracle.isprime1(v), v
        assert nt.factorize(v) and math.prod(p**e for p, e in nt.factorize(v).items()) == v


def test_carmichael_numbers_rejected():
    small = [561, 1105, 1729, 2465, 2821, 6601, 8911, 10585, 15841, 29341, 41041]
    big = []
    # Chernick: (6k+1)(12k+1)(18k+1) is a Carmichael number when all three are prime
    for k in range(1, 1 << 20):
        a, b, c = 6 * k + 1, 12 * k + 1, 18 * k + 1
        if a * b * c >= 1 << 64:
            break
        if nt.trial_is_prime(a) and nt.trial_is_prime(b) and nt.trial_is_prime(c):
            big.append(a * b * c)
    assert len(big) > 100
    for n in small + big:
        fac = nt.factorize(n)
        assert len(fac) >= 3 and all((n - 1) % (p - 1) == 0 for p in fac)  # Korselt
        assert not oracle.isprime1(n), n


def test_base2_strong_pseudoprimes_rejected():
    N = 10**6
    comp = ~nt.simple_sieve(N)
    found = [n for n in range(9, N, 2) if comp[n] and nt.strong_base2(n)]
    assert found[:5] == [2047, 3277, 4033, 4681, 8321]
    for n in found:
        assert oracle.sprp(n, 2)
        assert not oracle.isprime1(n)
    # constructed p*(2p-1) with p, 2p-1 prime near 2^31.5, kept if they pass base 2
    rng = random.Random(5)
    kept = 0
    while kept < 20:
        p = rng.randrange(2**31, 3_000_000_000) | 1  # p*(2p-1) < 2^64
        q = 2 * p - 1
        if nt.trial_is_prime(p) and nt.trial_is_prime(q) and nt.strong_base2(p * q):
            kept += 1
            assert oracle.sprp(p * q, 2)
            assert not oracle.isprime1(p * q)


def test_semiprimes_near_2p64_are_composite():
    small = load_pool("primes_near_2p32.txt").tolist()
    rng = random.Random(8)
    vals = [rng.choice(small) * rng.choice(small) for _ in range(2000)]
    out = oracle.isprime_u64(np.array(vals, dtype=np.uint64))
    assert not out.any()


def test_prime_pool_certificates():
    rng = random.Random(2)
    big = load_pool("primes_near_2p64.txt").tolist()
    for p in big[:100]:
        assert (1 << 64) - (1 << 40) <= p < 1 << 64
        assert nt.pratt_prime(p, rng)
    for p in load_pool("primes_near_2p32.txt").tolist()[:200]:
        assert nt.trial_is_prime(p)


def test_f64_domain():
    x = np.array([0.0, -0.0, 1.0, 2.0, 7.0, 9.0, 2.0**53, 2.0**53 - 111, float("nan"),
                  float("inf"), -float("inf"), -7.0, 2.5, 2.0**53 + 2, 1e300], dtype=np.float64)
    out, bad = oracle.isprime_f64(x)
    assert out.tolist() == [0, 0, 0, 1, 1, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0]
    assert bad == 7


# ---------------------------------------------------------------- workloads

def test_plain_small_prime_density():
    v = plain_small()
    out = oracle.isprime_u64(v)
    # independent check: the numpy sieve below 10^6
    ref = nt.simple_sieve(10**6)[v.astype(np.int64)]
    assert np.array_equal(out.astype(bool), ref)


def test_work_counter_invariants():
    v = plain_large(1 << 14)
    w = oracle.work_counts(v, td_bound=53)
    out = oracle.isprime_u64(v)
    assert w["primes"] == int(out.sum())
    # every prime passes base 2 and runs the other six bases; each composite
    # that reaches the test fails at exactly one base
    assert w["base2_passes"] >= w["primes"]
    assert w["base_tests"] >= w["mr64_elements"] + 6 * w["primes"]
    # binary schedule: fewer than 64 squarings and 64 multiplies per base test
    assert w["base2_squarings"] < 64 * w["mr64_elements"]
    assert w["rest_squarings"] < 64 * 6 * w["base2_passes"]
    assert w["base2_doublings"] < w["base2_squarings"]
    # trial division: 15 odd primes <= 53 for each odd element
    odd = int((v & np.uint64(1)).sum())
    assert w["trial_tests"] == 15 * odd


@pytest.mark.parametrize("bound", [53, 173, 239, 311, 457, 499])
def test_work_counter_trial_bound(bound):
    """The trial stage follows td_bound up to the end of the counter's list
    (499): every odd n >= 2^32 is tested against each odd prime <= td_bound
    (counted here by plain trial division of the small numbers), and n = p q
    (p the largest odd prime <= td_bound, q a prime near 2^50 found by the
    independent Pratt certificate) is removed at that bound and reaches the
    base-2 test one prime below it, failing there (checked by Python's pow)."""
    odd = [p for p in range(3, bound + 1, 2) if nt.trial_is_prime(p)]
    p = odd[-1]
    q = (1 << 50) + 1
    while nt.pratt_prime(q, random.Random(q)) is not True:
        q += 2
    n = p * q
    w = oracle.work_counts(np.array([n], dtype=np.uint64), td_bound=bound)
    assert w["trial_tests"] == len(odd)
    assert w["mr64_elements"] == 0 and w["base_tests"] == 0
    w = oracle.work_counts(np.array([n], dtype=np.uint64), td_bound=p - 1)
    assert w["trial_tests"] == len(odd) - 1
    assert w["mr64_elements"] == 1
    assert not nt.strong_base2(n)
    assert w["base2_passes"] == 0 and w["base_tests"] == 1


def test_work_counter_exact_on_one_prime():
    """n = 2^61 - 1: n - 1 = 2 (2^60 - 1), s = 1, d = 2^60 - 1 (60 one bits):
    every base does 59 squarings and 59 multiplications, no extra squaring."""
    w = oracle.work_counts(np.array([2**61 - 1], dtype=np.uint64), td_bound=53)
    assert w["mr64_elements"] == 1 and w["base2_passes"] == 1 and w["primes"] == 1
    assert w["base2_squarings"] == 59 and w["base2_doublings"] == 59
    assert w["rest_squarings"] == 6 * 59 and w["rest_multiplies"] == 6 * 59
    assert w["base_tests"] == 7 and w["trial_tests"] == 15


def test_work_counter_exact_fermat_f5():
    """n = F5 = 2^32 + 1 = 641 * 6700417 (no factor <= 53): n - 1 = 2^32, so
    s = 32 and d = 1.  Base 2: a^d = 2 needs no squaring or multiplication,
    then the tail squares 2 -> 4 -> 16 -> 256 -> 65536 -> 2^32 = -1 (mod n):
    exactly 5 squarings, and F5 passes base 2 (a base-2 strong pseudoprime)."""
    w = oracle.work_counts(np.array([2**32 + 1], dtype=np.uint64), td_bound=53)
    assert w["trial_tests"] == 15 and w["mr64_elements"] == 1
    assert w["base2_squarings"] == 5 and w["base2_doublings"] == 0
    assert w["base2_passes"] == 1 and w["primes"] == 0
    # the other bases: d = 1 again, so their whole work is tail squarings, at
    # most s - 1 = 31 per base, and the composite fails at one of them
    assert w["rest_multiplies"] == 0
    assert 2 <= w["base_tests"] <= 7
    assert w["rest_squarings"] <= 31 * (w["base_tests"] - 1)


def test_work_counter_exact_composite_full_tail():
    """n = 2^40 + 1 = 257 * 4278255361 (no factor <= 53): s = 40, d = 1.  The
    order of 2 mod n is 80 (2^40 = -1), and 2^(2^r) = -1 would need
    2^r = 40 (mod 80), = 1 would need 2^r = 0 (mod 80); neither happens, so
    the tail runs all s - 1 = 39 squarings and n fails base 2 there."""
    w = oracle.work_counts(np.array([2**40 + 1], dtype=np.uint64), td_bound=53)
    assert w["mr64_elements"] == 1 and w["base_tests"] == 1
    assert w["base2_squarings"] == 39 and w["base2_doublings"] == 0
    assert w["base2_passes"] == 0 and w["rest_squarings"] == 0 and w["primes"] == 0


def test_work_counter_exact_prime_s2():
    """p = 2^40 + 141 = 1099511627917 is prime (certificate below) with
    p = 5 (mod 8): s = 2 and d = (p - 1)/4 = 2^38 + 35 = 2^38 + 2^5 + 2 + 1,
    so each base's a^d takes bitlen(d) - 1 = 38 squarings and popcount(d) - 1
    = 3 multiplications.  With s = 2, a^(2d) = a^((p-1)/2) is the Legendre
    symbol (a/p) (Euler's criterion): for (a/p) = -1 the tail squares once
    and meets -1 (a^d is not +-1, its square being -1); for (a/p) = +1,
    a^d = +-1 and the tail is empty.  2 is a non-residue mod p = 5 (mod 8)."""
    p = 2**40 + 141
    assert nt.pratt_prime(p) and p % 8 == 5
    w = oracle.work_counts(np.array([p], dtype=np.uint64), td_bound=53)
    assert w["primes"] == 1 and w["base2_passes"] == 1 and w["base_tests"] == 7
    assert w["base2_squarings"] == 38 + 1 and w["base2_doublings"] == 3
    bases = [325, 9375, 28178, 450775, 9780504, 1795265022]
    nonres = sum(1 for a in bases if pow(a, (p - 1) // 2, p) == p - 1)
    assert w["rest_squarings"] == 6 * 38 + nonres
    assert w["rest_multiplies"] == 6 * 3
