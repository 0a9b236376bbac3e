"""Writes tests/golden/work_counts.json: the algorithmic work per element of
the benchmark workloads, counted by the CPU oracle's work counter.

The counter replays the method's schedule on every element (trial division
by the odd primes <= 53 for odd n >= 2^32, then the strong test to the bases
of Eq. 4 in order until one fails, each a^d by left-to-right binary
square-and-multiply as in Sec. 2.4, then the squarings of the strong test's
tail) and counts the modular operations.  The benchmark turns these counts
into the integer-pipe work of its roofline.  Nothing here touches the CUDA
library.

  plain_large  2^24 values (seed 1), every element
  batched      the 4096 ragged arrays (seed 3, 293,037,204 values), every element
  served_pool  the 2^27-value pool (seed 4) that the served benchmark slices
               its requests from, every element

Run from the repository root (about ten minutes on eight cores):
    python tests/golden/make_work_counts.py
"""
import concurrent.futures as cf
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import generators as g  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "work_counts.json")
CHUNK = 1 << 20


def count(values: np.ndarray, threads: int) -> dict:
    """oracle.work_counts over the whole array, in chunks on a thread pool
    (the ctypes call releases the interpreter lock)."""
    chunks = [values[i:i + CHUNK] for i in range(0, values.size, CHUNK)]
    total = dict.fromkeys(oracle.WORK_KEYS, 0)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for w in ex.map(lambda c: oracle.work_counts(c, td_bound=53, sieve_limit=1 << 32), chunks):
            for k, v in w.items():
                total[k] += v
    return total


def main():
    threads = os.cpu_count() or 1
    sets = {
        "plain_large": (lambda: g.plain_large(), g.WORKLOADS["plain_large"]),
        "batched": (lambda: g.batched_arrays()[0], g.WORKLOADS["batched"]),
        "served_pool": (lambda: g._replace_with_pools(g.bitlen_uniform(4, 1 << 27, 2, 64), 4),
                        "the 2^27 values (seed 4) the served benchmark slices its requests from: "
                        + g.WORKLOADS["served"]),
    }
    out = {"_about": "per-element means of the oracle's work counter (trial division by the "
                     "odd primes <= 53, sieve limit 2^32, bases of Eq. 4 in order, binary "
                     "left-to-right schedule); written by tests/golden/make_work_counts.py"}
    for name, (make, desc) in sets.items():
        v = make()
        w = count(v, threads)
        out[name] = {"elements": int(v.size), "description": desc,
                     "per_element": {k: w[k] / v.size for k in oracle.WORK_KEYS},
                     "totals": w}
        print(name, v.size, {k: round(w[k] / v.size, 4) for k in oracle.WORK_KEYS}, flush=True)
        del v
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
