"""Writes the prime pools used by the batched and served workloads.

Candidates are drawn with the seeded splitmix64 stream of the `workloads`
package; each is kept iff the CPU oracle declares it prime.  Nothing here
touches the CUDA library.

  primes_near_2p64.txt  4096 distinct primes in [2^64 - 2^40, 2^64)
  primes_near_2p32.txt  4096 distinct primes in [2^32 - 2^24, 2^32)

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
