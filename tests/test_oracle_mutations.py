"""Plants plausible mistakes in a copy of the oracle and checks the pins fail.

Each mutant is the oracle source with one textual change (a dropped term, an
off-by-one bound, a transposed operand, a missing overflow fix), compiled on
the CPU into a temporary library.  A battery of independent checks (the same
kinds of pins as test_oracle_pins.py, at smaller sizes) must reject every
mutant, and must accept the unmutated source.
"""
import ctypes
import math
import os
import random
import subprocess

import numpy as np
import pytest

import numtheory as nt

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "isprime_oracle.c")

MUTANTS = {
    "drop_minus_one_check": ("if (x == 1 || x == n - 1) return 1;", "if (x == 1) return 1;"),
    "short_squaring_loop": ("for (int r = 1; r < s; ++r) {", "for (int r = 1; r < s - 1; ++r) {"),
    "trial_bound_strict": ("for (uint64_t d = 3; d * d <= n; d += 2)",
                           "for (uint64_t d = 3; d * d < n; d += 2)"),
    "transposed_multiply": ("r = oracle_mulmod(r, a, m);", "r = oracle_mulmod(a, a, m);"),
    "wrong_s": ("int s = __builtin_ctzll(d);", "int s = __builtin_ctzll(d) - 1;"),
    "doubling_overflow": ("a = oracle_modadd(a, a, m);", "a = (a << 1) % m;"),
    "modadd_strict": ("return (a >= gap) ? a - gap : a + b;", "return (a > gap) ? a - gap : a + b;"),
    "f64_limit_strict": ("!(x <= lim)", "!(x < lim)"),
    "small_prime_equal": ("if (n % kSmallPrimes[i] == 0) return 0;",
                          "if (n % kSmallPrimes[i] == 1) return 0;"),
    "leading_bit_skipped": ("r = a; /* the leading 1 bit */", "r = 1 % m; /* the leading 1 bit */"),
    "n_minus_one_wrong_sign": ("if (x == n - 1) return 1;", "if (x == n + 1) return 1;"),
}


def _build(src_text, tmp_path, name):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so),
                    str(c), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    u64, p, sz = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
    L.oracle_isprime1.argtypes = [u64]
    L.oracle_isprime1.restype = ctypes.c_int
    L.oracle_isprime_u64.argtypes = [p, p, sz]
    L.oracle_mulmod_classic.argtypes = [u64, u64, u64]
    L.oracle_mulmod_classic.restype = u64
    L.oracle_modadd.argtypes = [u64, u64, u64]
    L.oracle_modadd.restype = u64
    L.oracle_isprime_f64.argtypes = [p, p, sz]
    L.oracle_isprime_f64.restype = u64
    L.oracle_sprp.argtypes = [u64, u64]
    L.oracle_sprp.restype = ctypes.c_int
    return L


def _classify(L, vals):
    a = np.ascontiguousarray(vals, dtype=np.uint64)
    out = np.empty(a.size, dtype=np.uint8)
    L.oracle_isprime_u64(a.ctypes.data, out.ctypes.data, a.size)
    return out.astype(bool)


_CACHE = {}


def _battery_expectations():
    if not _CACHE:
        _CACHE["small"] = nt.simple_sieve(200_000)
        lo = 1 << 32
        _CACHE["w32"] = (lo, nt.window_sieve(lo, lo + (1 << 18)))
        lo = (1 << 40) - (1 << 16)
        _CACHE["w40"] = (lo, nt.window_sieve(lo, lo + (1 << 17)))
        comp = ~nt.simple_sieve(10**6)
        _CACHE["spsp"] = [n for n in range(9, 10**6, 2) if comp[n] and nt.strong_base2(n)]
        _CACHE["sprp2"] = [(n, nt.strong_base2(n)) for n in range(3, 60_000, 2)]
    return _CACHE


def _battery(L):
    """Returns the list of failed check names (empty = all pins hold)."""
    e = _battery_expectations()
    failed = []
    if not np.array_equal(_classify(L, np.arange(200_001)), e["small"]):
        failed.append("sieve<2e5")
    lo, ref = e["w32"]
    if not np.array_equal(_classify(L, np.arange(lo, lo + ref.size, dtype=np.uint64)), ref):
        failed.append("window@2^32")
    lo, ref = e["w40"]
    if not np.array_equal(_classify(L, np.arange(lo, lo + ref.size, dtype=np.uint64)), ref):
        failed.append("window@2^40")
    if _classify(L, e["spsp"]).any():
        failed.append("strong pseudoprimes")
    if any(bool(L.oracle_sprp(n, 2)) != f for n, f in e["sprp2"]):
        failed.append("base-2 strong test")
    known = [2**31 - 1, 2**32 - 5, 2**61 - 1, 2**63 - 25, 2**64 - 59]
    if not _classify(L, known).all():
        failed.append("known primes")
    rng = random.Random(4)
    for m in [2**64 - 59, 2**64 - 1, 2**63 + 1] + [rng.randrange(3, 2**64) for _ in range(50)]:
        for a, b in [(m - 1, m - 1), (m - 1, 1)] + [(rng.randrange(m), rng.randrange(m))
                                                    for _ in range(10)]:
            if L.oracle_mulmod_classic(a, b, m) != a * b % m or L.oracle_modadd(a, b, m) != (a + b) % m:
                failed.append("mulmod")
                break
        else:
            continue
        break
    x = np.array([2.0**53, 7.0, float("nan"), -1.0], dtype=np.float64)
    out = np.empty(4, dtype=np.uint8)
    bad = L.oracle_isprime_f64(x.ctypes.data, out.ctypes.data, 4)
    if bad != 2 or out.tolist() != [0, 1, 0, 0]:
        failed.append("f64")
    return failed


def test_unmutated_source_passes(tmp_path):
    L = _build(open(SRC).read(), tmp_path, "orig")
    assert _battery(L) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    L = _build(src.replace(old, new), tmp_path, name)
    assert _battery(L), f"mutant {name} survived every pin"


# Mistakes in the work counter alone (the primality results stay right, so
# only the exact counts of test_oracle_pins.py can see them).
WORK_MUTANTS = {
    "tail_squaring_not_counted": ("    x = oracle_mulmod(x, x, n);\n    if (sq) ++*sq;",
                                  "    x = oracle_mulmod(x, x, n);"),
    "multiply_counted_as_squaring": ("      if (mu) ++*mu;", "      if (sq) ++*sq;"),
    "base_counts_start_at_one": ("uint64_t sq = 0, mu = 0;", "uint64_t sq = 1, mu = 0;"),
    "trial_bound_exclusive": ("odd_primes[k] <= td_bound", "odd_primes[k] < td_bound"),
}

WORK_KEYS = ("mr64_elements", "base2_squarings", "base2_doublings", "base2_passes",
             "rest_squarings", "rest_multiplies", "base_tests", "trial_tests",
             "mr32_elements", "primes")


def _work(L, n):
    a = np.array([n], dtype=np.uint64)
    c = np.zeros(len(WORK_KEYS), dtype=np.uint64)
    L.oracle_work_counts(a.ctypes.data, 1, 53, 1 << 32, c.ctypes.data)
    return dict(zip(WORK_KEYS, (int(x) for x in c)))


def _work_battery(L):
    """The exact counts pinned by hand in test_oracle_pins.py."""
    L.oracle_work_counts.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_void_p]
    L.oracle_work_counts.restype = None
    failed = []
    w = _work(L, 2**32 + 1)
    if (w["base2_squarings"], w["base2_doublings"], w["trial_tests"]) != (5, 0, 15):
        failed.append("F5")
    w = _work(L, 2**40 + 1)
    if (w["base2_squarings"], w["base_tests"]) != (39, 1):
        failed.append("2^40+1")
    w = _work(L, 2**61 - 1)
    if (w["base2_squarings"], w["base2_doublings"], w["rest_squarings"],
            w["rest_multiplies"]) != (59, 59, 354, 354):
        failed.append("2^61-1")
    p = 2**40 + 141
    nonres = sum(1 for a in [325, 9375, 28178, 450775, 9780504, 1795265022]
                 if pow(a, (p - 1) // 2, p) == p - 1)
    w = _work(L, p)
    if (w["base2_squarings"], w["base2_doublings"], w["rest_squarings"],
            w["rest_multiplies"]) != (39, 3, 228 + nonres, 18):
        failed.append("2^40+141")
    return failed


def test_unmutated_counter_passes(tmp_path):
    L = _build(open(SRC).read(), tmp_path, "orig_work")
    assert _work_battery(L) == []


@pytest.mark.parametrize("name", sorted(WORK_MUTANTS))
def test_counter_mutant_is_caught(tmp_path, name):
    old, new = WORK_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    L = _build(src.replace(old, new), tmp_path, "w_" + name)
    assert _work_battery(L), f"counter mutant {name} survived every exact count"
