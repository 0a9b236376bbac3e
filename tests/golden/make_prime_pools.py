"""Writes the prime pools used by the batched and served workloads.

Candidates are drawn with the seeded splitmix64 stream of the `workloads`
package; each is kept iff the CPU oracle declares it prime.  Nothing here
touches the CUDA library.

  primes_near_2p64.txt  4096 distinct primes in [2^64 - 2^40, 2^64)
  primes_near_2p32.txt  4096 distinct primes in [2^32 - 2^24, 2^32)
  primes_by_bits.txt    100 random primes of each bit size of Table 4 (4 ... 64
                        bits, i.e. in [2^(b-1), 2^b)), drawn with replacement

Run from the repository root:  python tests/golden/make_prime_pools.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads.generators import uniform_range  # noqa: E402


def pool(lo, hi, count, seed):
    got = []
    seen = set()
    offset = 0
    while len(got) < count:
        cand = uniform_range(seed, 1 << 16, lo, hi, offset=offset) | np.uint64(1)
        offset += 1 << 16
        flags = oracle.isprime_u64(cand)
        for v, f in zip(cand.tolist(), flags.tolist()):
            if f and v not in seen:
                seen.add(v)
                got.append(v)
                if len(got) == count:
                    break
    return got


T4_BITS = (4, 8, 16, 24, 32, 36, 40, 44, 48, 50, 52, 56, 60, 64)


def primes_of_bits(b, count, seed):
    """`count` primes in [2^(b-1), 2^b), uniform candidates, repeats allowed."""
    got = []
    offset = 0
    while len(got) < count:
        cand = uniform_range(seed, 1 << 12, 1 << (b - 1), 1 << b, offset=offset)
        offset += 1 << 12
        flags = oracle.isprime_u64(cand)
        got.extend(v for v, f in zip(cand.tolist(), flags.tolist()) if f)
    return got[:count]


def write(name, vals, header):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        f.write(f"# {header}\n# written by tests/golden/make_prime_pools.py (CPU oracle)\n")
        for v in vals:
            f.write(f"{v:016x}\n")


if __name__ == "__main__":
    write("primes_near_2p64.txt", pool((1 << 64) - (1 << 40), 1 << 64, 4096, 64),
          "4096 distinct primes in [2^64 - 2^40, 2^64), hex")
    write("primes_near_2p32.txt", pool((1 << 32) - (1 << 24), 1 << 32, 4096, 32),
          "4096 distinct primes in [2^32 - 2^24, 2^32), hex")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "primes_by_bits.txt")
    with open(path, "w") as f:
        f.write("# 100 random primes of each bit size b of Table 4, in [2^(b-1), 2^b): "
                "bits hex\n# written by tests/golden/make_prime_pools.py (CPU oracle)\n")
        for b in T4_BITS:
            for v in primes_of_bits(b, 100, 1000 + b):
                f.write(f"{b} {v:016x}\n")
