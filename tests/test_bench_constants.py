"""The per-element work figures bench.py uses for the roofline are what the
oracle's work counter measures on the benchmark's array.  CPU only."""
import os
import sys

import numpy as np

import oracle
from workloads import plain_large

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_plain_large_work_per_element():
    v = plain_large()
    w = oracle.work_counts(v, td_bound=53, sieve_limit=1 << 32)
    for k, per in bench.WORK_PLAIN_LARGE.items():
        assert abs(w[k] / v.size - per) < 1e-4, (k, w[k] / v.size, per)


def test_bench_workload_is_the_generator_array():
    v, _ = bench._workload("plain_large", 0)
    assert np.array_equal(v, plain_large())
