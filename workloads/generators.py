"""Counter-based splitmix64 generators for the five workloads.

splitmix64 (Steele, Lea, Flood 2014): the i-th output of stream `seed` is
mix(seed * 2^64/phi + (i + 1) * 0x9E3779B97F4A7C15) with the published
finaliser constants.  Vectorised in numpy with wrapping uint64 arithmetic.

Workloads (each with the shapes and value distributions of the paper's array
experiments, Sec. 6 and Sec. 8.2 / Table 5, scaled to the GPU):
  plain_small   100,000 values uniform in [0, 10^6), seed 0
  plain_large   2^24 values uniform in [2^49, 2^64), even indices forced odd
  plain_mixed   2^26 values, bit length uniform in 2..64, value uniform within
                that bit length; plus 2^20 doubles holding integers uniform in
                [0, 2^53)
  batched       4096 ragged arrays, sizes log-uniform in 1..2^20, values as
                plain_mixed, 25% replaced by primes near 2^64 and 10% by
                semiprimes p*q with p, q near 2^32 (pools from tests/golden)
  served        20,000 requests, exponential inter-arrival (mean 200 us),
                sizes log-uniform in 1..2^22, values as batched
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)

_POOL_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         "tests", "golden")


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive outputs (starting at index `offset`) of stream `seed`."""
    with np.errstate(over="ignore"):
        base = np.uint64((seed * GOLDEN) & 0xFFFFFFFFFFFFFFFF)
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = base + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _mulhi64(a: np.ndarray, b) -> np.ndarray:
    """High 64 bits of the 128-bit product a*b (elementwise, exact)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.broadcast_to(np.asarray(b, dtype=np.uint64), a.shape)
    s32 = np.uint64(32)
    a0, a1 = a & _MASK32, a >> s32
    b0, b1 = b & _MASK32, b >> s32
    with np.errstate(over="ignore"):
        p00 = a0 * b0
        p01 = a0 * b1
        p10 = a1 * b0
        p11 = a1 * b1
        mid = (p00 >> s32) + (p01 & _MASK32) + (p10 & _MASK32)
        return p11 + (p01 >> s32) + (p10 >> s32) + (mid >> s32)


def uniform_below(r: np.ndarray, bound) -> np.ndarray:
    """Map uniform 64-bit r to [0, bound) by the high half of r*bound."""
    return _mulhi64(r, bound)


def uniform_range(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """n values uniform in [lo, hi), hi <= 2^64."""
    r = splitmix64(seed, n, offset)
    span = hi - lo
    if span >= 1 << 64:
        return r
    with np.errstate(over="ignore"):
        return np.uint64(lo) + uniform_below(r, np.uint64(span))


def bitlen_uniform(seed: int, n: int, lo_bits: int = 2, hi_bits: int = 64,
                   offset: int = 0) -> np.ndarray:
    """Bit length uniform in lo_bits..hi_bits, value uniform within it."""
    r1 = splitmix64(seed, n, offset)
    r2 = splitmix64(seed ^ 0x5DEECE66D, n, offset)
    nb = np.uint64(hi_bits - lo_bits + 1)
    b = uniform_below(r1, nb) + np.uint64(lo_bits)          # bit length
    half = np.left_shift(np.uint64(1), b - np.uint64(1))    # 2^(b-1)
    with np.errstate(over="ignore"):
        return half + uniform_below(r2, half)


def log_uniform_sizes(seed: int, n: int, max_size: int) -> np.ndarray:
    """floor(exp(U * ln(max_size + 1))) clamped to [1, max_size]."""
    r = splitmix64(seed, n)
    u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    s = np.floor(np.exp(u * np.log(max_size + 1.0))).astype(np.int64)
    return np.clip(s, 1, max_size)


def load_pool(name: str) -> np.ndarray:
    """Stored prime pools (written by tests/golden/make_prime_pools.py)."""
    path = os.path.join(_POOL_DIR, name)
    vals = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 16))
    return np.array(vals, dtype=np.uint64)


def load_primes_by_bits() -> dict:
    """bits -> uint64 array of the stored primes of that bit size (Table 4's
    scalar inputs; written by tests/golden/make_prime_pools.py)."""
    out: dict = {}
    with open(os.path.join(_POOL_DIR, "primes_by_bits.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                b, v = line.split()
                out.setdefault(int(b), []).append(int(v, 16))
    return {b: np.array(v, dtype=np.uint64) for b, v in out.items()}


# --- the five workloads --------------------------------------------------

def plain_small(n: int = 100_000, seed: int = 0) -> np.ndarray:
    return uniform_range(seed, n, 0, 10**6)


def plain_large(n: int = 1 << 24, seed: int = 1) -> np.ndarray:
    v = uniform_range(seed, n, 1 << 49, 1 << 64)
    v[0::2] |= np.uint64(1)
    return v


def plain_mixed(n: int = 1 << 26, seed: int = 2, offset: int = 0) -> np.ndarray:
    return bitlen_uniform(seed, n, 2, 64, offset)


def mixed_doubles(n: int = 1 << 20, seed: int = 2) -> np.ndarray:
    r = splitmix64(seed ^ 0xD0B1E, n)
    return (r >> np.uint64(11)).astype(np.float64)


def _replace_with_pools(v: np.ndarray, seed: int, offset: int = 0) -> np.ndarray:
    """v holds the stream's values at indices offset .. offset + v.size - 1."""
    n = v.size
    big = load_pool("primes_near_2p64.txt")
    small = load_pool("primes_near_2p32.txt")
    r = splitmix64(seed ^ 0xBA7C4, n, offset)
    u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    pick = splitmix64(seed ^ 0x9001, n, offset)
    pick2 = splitmix64(seed ^ 0x9002, n, offset)
    is_p = u < 0.25
    is_sp = (u >= 0.25) & (u < 0.35)
    v = v.copy()
    v[is_p] = big[uniform_below(pick[is_p], np.uint64(big.size)).astype(np.int64)]
    p = small[uniform_below(pick[is_sp], np.uint64(small.size)).astype(np.int64)]
    q = small[uniform_below(pick2[is_sp], np.uint64(small.size)).astype(np.int64)]
    with np.errstate(over="ignore"):
        v[is_sp] = p * q  # p, q < 2^32, so p*q < 2^64 exactly
    return v


def batched_arrays(n_arrays: int = 4096, max_size: int = 1 << 20, seed: int = 3):
    """Returns (values concatenated, offsets[n_arrays+1])."""
    sizes = log_uniform_sizes(seed, n_arrays, max_size)
    offsets = np.zeros(n_arrays + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    v = bitlen_uniform(seed, int(offsets[-1]), 2, 64)
    return _replace_with_pools(v, seed), offsets


def served_requests(n_requests: int = 20_000, max_size: int = 1 << 22,
                    rate_per_s: float = 5000.0, seed: int = 4,
                    values: bool = True):
    """Returns (arrival_times_s, sizes, values-or-None).

    Arrivals are a Poisson process: exponential gaps with mean 1/rate."""
    sizes = log_uniform_sizes(seed, n_requests, max_size)
    r = splitmix64(seed ^ 0xA331, n_requests)
    u = ((r >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    gaps = -np.log(u) / rate_per_s
    arrivals = np.cumsum(gaps)
    vals = None
    if values:
        total = int(sizes.sum())
        vals = _replace_with_pools(bitlen_uniform(seed, total, 2, 64), seed)
    return arrivals, sizes, vals


WORKLOADS = {
    "plain_small": "100,000 uint64 uniform in [0, 10^6), seed 0",
    "plain_large": "2^24 uint64 uniform in [2^49, 2^64), even indices forced odd, seed 1",
    "plain_mixed": "2^26 uint64 with bit length uniform in 2..64 (+2^20 f64 in [0, 2^53)), seed 2",
    "batched": "4096 ragged arrays, log-uniform sizes 1..2^20, mixed values, 25% primes near 2^64, "
               "10% semiprimes near 2^64, seed 3",
    "served": "20,000 Poisson requests at 5,000 req/s, log-uniform sizes 1..2^22, values as batched, seed 4",
}
