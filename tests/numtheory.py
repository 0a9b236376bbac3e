"""Independent number theory used to pin the oracle (tests only).

Nothing here shares code with the oracle or the CUDA library: plain Python
integers and numpy, different algorithms (sieves, Pollard-Brent rho, Lucas
/ Pratt certificates) from the Miller-Rabin the oracle runs.
"""
from __future__ import annotations

import math
import random

import numpy as np


def simple_sieve(limit: int) -> np.ndarray:
    """Boolean array is_prime[0..limit] by the sieve of Eratosthenes."""
    s = np.ones(limit + 1, dtype=bool)
    s[:2] = False
    for p in range(2, math.isqrt(limit) + 1):
        if s[p]:
            s[p * p::p] = False
    return s


def window_sieve(lo: int, hi: int) -> np.ndarray:
    """is_prime for the integers lo..hi-1 (segmented sieve; hi^(1/2) small)."""
    n = hi - lo
    flags = np.ones(n, dtype=bool)
    base = np.flatnonzero(simple_sieve(math.isqrt(hi - 1) + 1))
    for p in base.tolist():
        start = max(p * p, ((lo + p - 1) // p) * p)
        if start >= hi:
            continue
        flags[start - lo::p] = False
    for v in (0, 1):
        if lo <= v < hi:
            flags[v - lo] = False
    return flags


def trial_is_prime(n: int) -> bool:
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    d = 3
    while d * d <= n:
        if n % d == 0:
            return False
        d += 2
    return True


def pollard_brent(n: int, rng: random.Random) -> int:
    """A nontrivial factor of composite n (n odd, not a prime power of 2)."""
    if n % 2 == 0:
        return 2
    for p in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return p
    while True:
        y, c, m = rng.randrange(1, n), rng.randrange(1, n), 128
        g = r = q = 1
        while g == 1:
            x = y
            for _ in range(r):
                y = (y * y + c) % n
            k = 0
            while k < r and g == 1:
                ys = y
                for _ in range(min(m, r - k)):
                    y = (y * y + c) % n
                    q = q * abs(x - y) % n
                g = math.gcd(q, n)
                k += m
            r *= 2
        if g == n:
            g = 1
            while g == 1:
                ys = (ys * ys + c) % n
                g = math.gcd(abs(x - ys), n)
        if g != n:
            return g


def _small_factor(n: int, bound: int = 1000):
    for p in range(2, min(bound, math.isqrt(n)) + 1):
        if n % p == 0:
            return p
    return None


def factorize(n: int, rng: random.Random | None = None) -> dict:
    """Prime factorisation {p: e}; primality of each factor is proved by a
    Pratt certificate (factors above 2^20) or trial division."""
    rng = rng or random.Random(12345)
    out: dict = {}
    stack = [n]
    while stack:
        m = stack.pop()
        if m == 1:
            continue
        if m < (1 << 20):
            f = _small_factor(m, math.isqrt(m) + 1)
            if f is None:
                out[m] = out.get(m, 0) + 1
            else:
                stack += [f, m // f]
            continue
        f = _small_factor(m)
        if f is not None:
            stack += [f, m // f]
            continue
        if pratt_prime(m, rng) is True:
            out[m] = out.get(m, 0) + 1
            continue
        f = pollard_brent(m, rng)
        stack += [f, m // f]
    return out


def _fermat_composite(n: int) -> bool:
    """True if some small base proves n composite by Fermat (cheap filter)."""
    for a in (2, 3, 5, 7, 11, 13):
        if a % n and pow(a, n - 1, n) != 1:
            return True
    return False


def pratt_prime(n: int, rng: random.Random | None = None):
    """Proves n prime with a Lucas certificate, recursively.

    Brillhart-Lehmer-Selfridge form of Lucas's theorem: if for every prime
    q | n-1 some a_q has a_q^(n-1) = 1 and a_q^((n-1)/q) != 1 (mod n), then n
    is prime.  Returns True (proved prime), False (shown composite: a Fermat
    witness), or None (no certificate found; the caller factors n instead)."""
    rng = rng or random.Random(54321)
    if n < (1 << 20):
        return trial_is_prime(n)
    if _fermat_composite(n):
        return False
    fac = factorize(n - 1, rng)
    for q in fac:
        for a in range(2, 400):
            if pow(a, n - 1, n) != 1:
                return False
            if pow(a, (n - 1) // q, n) != 1:
                break
        else:
            return None
    return True


def strong_base2(n: int) -> bool:
    """Strong probable prime to base 2, Python big integers."""
    if n < 3 or n % 2 == 0:
        return n == 2
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    x = pow(2, d, n)
    if x in (1, n - 1):
        return True
    for _ in range(s - 1):
        x = x * x % n
        if x == n - 1:
            return True
    return False


def jacobi(a: int, n: int) -> int:
    """Jacobi symbol (a/n), n odd positive (quadratic reciprocity, Python ints)."""
    a %= n
    t = 1
    while a:
        while a % 2 == 0:
            a //= 2
            if n % 8 in (3, 5):
                t = -t
        a, n = n, a
        if a % 4 == 3 and n % 4 == 3:
            t = -t
        a %= n
    return t if n == 1 else 0


def strong_lucas(n: int) -> bool:
    """Strong Lucas probable prime, Selfridge's method A (D = 5, -7, 9, ...,
    P = 1, Q = (1 - D)/4), from the Lucas sequences' definition with
    exact integer doubling formulas.  n odd, not a perfect square."""
    D = 5
    while jacobi(D, n) != -1:
        if jacobi(D, n) == 0 and abs(D) != n:
            return False
        D = -(D + 2) if D > 0 else -D + 2
    P, Q = 1, (1 - D) // 4
    d, s = n + 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    inv2 = (n + 1) // 2
    U, V, Qk = 1, P, Q % n
    for bit in bin(d)[3:]:
        U, V, Qk = U * V % n, (V * V - 2 * Qk) % n, Qk * Qk % n
        if bit == "1":
            U, V = (P * U + V) * inv2 % n, (D * U + P * V) * inv2 % n
            Qk = Qk * Q % n
    if U == 0 or V == 0:
        return True
    for _ in range(s - 1):
        V = (V * V - 2 * Qk) % n
        if V == 0:
            return True
        Qk = Qk * Qk % n
    return False
