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
  plain_large_td2
               plain_large under the two-stage trial division of the base-2
               kernel (tuning td2_groups = G in 8, 12, 16, 24): the first
               stage tests the odd primes <= 53 on every odd element, the
               second the next 3 G odd primes (up to P = 173, 239, 311, 457)
               on the first stage's survivors only.  Which elements reach the
               base-2 test, and everything after it, is the oracle's count at
               td_bound = P; the trial tests are the first stage's count at
               53 plus 3 G per survivor of the first stage.

Run from the repository root (about ten minutes on eight cores):
    python tests/golden/make_work_counts.py
or, to recompute some sets and keep the others:
    python tests/golden/make_work_counts.py plain_large_td2
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


TD2_BOUNDS = {8: 173, 12: 239, 16: 311, 24: 457}  # td2_groups -> largest prime of its groups


def count(values: np.ndarray, threads: int, td_bound: int = 53) -> dict:
    """oracle.work_counts over the whole array, in chunks on a thread pool
    (the ctypes call releases the interpreter lock)."""
    chunks = [values[i:i + CHUNK] for i in range(0, values.size, CHUNK)]
    total = dict.fromkeys(oracle.WORK_KEYS, 0)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for w in ex.map(lambda c: oracle.work_counts(c, td_bound=td_bound, sieve_limit=1 << 32),
                        chunks):
            for k, v in w.items():
                total[k] += v
    return total


def count_td2(values: np.ndarray, threads: int) -> dict:
    """Per td2_groups G: the two-stage schedule's counts (see the module
    docstring)."""
    first = count(values, threads, 53)
    out = {}
    for groups, bound in TD2_BOUNDS.items():
        w = count(values, threads, bound)
        w["trial_tests"] = first["trial_tests"] + 3 * groups * first["mr64_elements"]
        out[str(groups)] = {"td_bound": bound,
                            "per_element": {k: w[k] / values.size for k in oracle.WORK_KEYS},
                            "totals": w}
    return out


def main():
    threads = os.cpu_count() or 1
    sets = {
        "plain_large": (lambda: g.plain_large(), g.WORKLOADS["plain_large"]),
        "batched": (lambda: g.batched_arrays()[0], g.WORKLOADS["batched"]),
        "served_pool": (lambda: g._replace_with_pools(g.bitlen_uniform(4, 1 << 27, 2, 64), 4),
                        "the 2^27 values (seed 4) the served benchmark slices its requests from: "
                        + g.WORKLOADS["served"]),
        "plain_large_td2": (lambda: g.plain_large(),
                            "plain_large under the base-2 kernel's second trial stage, keyed by "
                            "td2_groups: " + g.WORKLOADS["plain_large"]),
    }
    only = sys.argv[1:] or list(sets)
    out = {}
    if os.path.exists(OUT) and sys.argv[1:]:
        with open(OUT) as f:
            out = json.load(f)
    out["_about"] = ("per-element means of the oracle's work counter (trial division by the "
                     "odd primes <= 53, sieve limit 2^32, bases of Eq. 4 in order, binary "
                     "left-to-right schedule; plain_large_td2: the two-stage trial division "
                     "of the base-2 kernel); written by tests/golden/make_work_counts.py")
    for name in only:
        make, desc = sets[name]
        v = make()
        if name == "plain_large_td2":
            out[name] = {"elements": int(v.size), "description": desc, "groups": count_td2(v, threads)}
            for grp, e in out[name]["groups"].items():
                print(name, grp, {k: round(x, 4) for k, x in e["per_element"].items()}, flush=True)
        else:
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
