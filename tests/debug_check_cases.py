"""Parity cases run under the debug build of the library (bounds checks
compiled in); executed by tests/test_gpu_debug_checks.py in a child process
whose ISPRIME_GB300_LIB names the debug library.  Prints one JSON line: the
cases run, the mismatches against the oracle, and the check record."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2108_04791_gb300 as ipg  # noqa: E402
from workloads import plain_large, plain_mixed, plain_small  # noqa: E402


def main():
    dev = torch.device("cuda:0")
    assert os.environ.get("ISPRIME_GB300_LIB", "").endswith("_dbg.so")
    before = ipg.debug_checks(reset=True)
    cases, bad = 0, []

    def check(name, vals, got):
        nonlocal cases
        cases += 1
        want = oracle.isprime_u64(vals)
        if not np.array_equal(got, want):
            bad.append(name)

    def dev_run(c, v):
        t = torch.from_numpy(np.ascontiguousarray(v).view(np.int64)).to(dev)
        out = c.isprime(t)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    with ipg.Context(0, sieve_limit=1 << 26) as c:
        v = np.concatenate([plain_small(20_000), plain_large(1 << 18, seed=3),
                            plain_mixed(1 << 18, seed=4)])
        for kw in (dict(), dict(td_fold=2, base2_split=1, base2_ilp=2, rest_window=3),
                   dict(base2_window=4), dict(base2_window=0), dict(rest_test=1),
                   dict(compact_min=8), dict(chunk_log2=16), dict(sieve_cutover_log2=20),
                   dict(small_max=1 << 20)):
            c.set_tuning(**{**dict(td_fold=0, base2_split=0, base2_ilp=1, rest_window=4,
                                   base2_window=1, rest_test=0, compact_min=33, chunk_log2=24,
                                   sieve_cutover_log2=32, small_max=0), **kw})
            check(f"plain {kw}", v, dev_run(c, v))
            check(f"ragged {kw}", v[1:40001], dev_run(c, v[1:40001]))
        c.set_tuning(small_max=0, chunk_log2=16)
        check("host path", v, c.isprime_host(v))
        parts = np.split(v, [1, 100, 5000, 70000])
        outs = c.isprime_batched([torch.from_numpy(p.view(np.int64)).to(dev) for p in parts])
        torch.cuda.synchronize()
        check("batched", v, np.concatenate([o.cpu().numpy() for o in outs]))
        for lo, cnt in ((1, 1 << 20), ((1 << 26) - 5000, 70_000), (2**64 - (1 << 18), 1 << 18)):
            out = c.isprime_range(lo, cnt)
            torch.cuda.synchronize()
            check(f"range {lo}", np.arange(cnt, dtype=np.uint64) + np.uint64(lo), out.cpu().numpy())
        rng = np.random.default_rng(1)
        w = (np.uint64(1 << 40) + rng.integers(0, 1 << 18, 1 << 18, dtype=np.uint64))
        c.set_tuning(window_ratio16=4096, chunk_log2=24)
        check("window path", w, dev_run(c, w))
        c.set_tuning(window_ratio16=0)
    torch.cuda.synchronize()
    after = ipg.debug_checks(reset=True)
    print(json.dumps({"cases": cases, "mismatches": bad, "before": before, "after": after}))


if __name__ == "__main__":
    main()
