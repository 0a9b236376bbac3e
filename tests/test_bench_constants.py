"""The per-element work figures bench.py uses for its rooflines are what the
oracle's work counter measures on the benchmark's inputs, and both arms of
the benchmark describe the workload with the same config.  CPU only."""
import json
import os
import subprocess
import sys

import numpy as np

import oracle
from workloads import generators as wg
from workloads import plain_large

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden", "work_counts.json")


def test_plain_large_work_per_element():
    v = plain_large()
    w = oracle.work_counts(v, td_bound=53, sieve_limit=1 << 32)
    for k, per in bench.WORK_PLAIN_LARGE.items():
        assert abs(w[k] / v.size - per) < 1e-4, (k, w[k] / v.size, per)
    g = json.load(open(GOLDEN))["plain_large"]
    assert g["totals"] == w and g["elements"] == v.size


def test_plain_large_two_stage_trial_work():
    """The stored counts of the base-2 kernel's second trial stage: at the
    larger trial bound fewer elements reach base 2, the same ones pass it (no
    prime is removed, and no base-2 strong pseudoprime of this array has a
    factor below 457), and the trial tests are the first stage's plus 3 G per
    first-stage survivor; a recount of every td_bound on 2^18 elements agrees
    within sampling error, and the bench reads the schedule from the tuning."""
    g = json.load(open(GOLDEN))
    base = g["plain_large"]["per_element"]
    v = plain_large(1 << 18)
    for groups, bound in ((8, 173), (12, 239), (16, 311), (24, 457)):
        e = g["plain_large_td2"]["groups"][str(groups)]
        per = e["per_element"]
        assert e["td_bound"] == bound
        assert per["mr64_elements"] < base["mr64_elements"]
        assert per["base2_squarings"] < base["base2_squarings"]
        assert per["base2_passes"] == base["base2_passes"] and per["primes"] == base["primes"]
        assert abs(per["trial_tests"] - (base["trial_tests"] + 3 * groups * base["mr64_elements"])) < 1e-9
        w = oracle.work_counts(v, td_bound=bound, sieve_limit=1 << 32)
        for k in ("mr64_elements", "base2_squarings"):
            assert abs(w[k] / v.size - per[k]) < 0.02 * per[k], (groups, k)
        work, stage2, sched = bench._plain_large_work({"td2_groups": groups})
        assert work == per and abs(stage2 - 3 * groups * bench.WORK_PLAIN_LARGE["mr64_elements"]) < 1e-12
        assert str(bound) in sched
    work, stage2, _ = bench._plain_large_work({"td2_groups": 0})
    assert work == bench.WORK_PLAIN_LARGE and stage2 == 0


def test_ncu_traffic_is_recorded_for_the_default_tuning():
    """bench.py reports the ncu DRAM bytes only for the build and tuning the
    capture was taken with; the recorded tuning must be the library's
    defaults (the bench runs them), else every line would carry null.  (The
    source hash is compared at run time: a kernel changed after the capture
    gives null until the next capture.)"""
    import paper_2108_04791_gb300 as ipg
    assert bench.NCU_TRAFFIC["tuning"] == ipg.default_tuning()
    assert len(bench.NCU_TRAFFIC["sources"]) == 16


def test_batched_and_served_work_on_a_sample():
    """The stored full-workload figures (written by make_work_counts.py over
    every element) agree with a recount of 2^18 elements taken in 16 blocks
    spread over each workload, within sampling error."""
    g = json.load(open(GOLDEN))
    for name, seed, total in (("batched", 3, g["batched"]["elements"]),
                              ("served_pool", 4, g["served_pool"]["elements"])):
        assert total == (293_037_204 if name == "batched" else 1 << 27)
        parts = []
        for k in range(16):
            off = (total // 16) * k
            v = wg.bitlen_uniform(seed, 1 << 14, 2, 64, offset=off)
            parts.append(wg._replace_with_pools(v, seed, off))
        v = np.concatenate(parts)
        w = oracle.work_counts(v, td_bound=53, sieve_limit=1 << 32)
        per = g[name]["per_element"]
        for k in ("base2_squarings", "rest_squarings", "rest_multiplies", "trial_tests"):
            got = w[k] / v.size
            assert abs(got - per[k]) < 0.05 * per[k] + 0.05, (name, k, got, per[k])
    # the slots per element the bench derives from them
    s = bench._slots_per_element(g["batched"]["per_element"])
    assert 2500 < s < 3700


def test_both_arms_print_the_same_config(tmp_path):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    v, desc = bench._workload("plain_large", 0)
    assert line["config"] == bench._config("plain_large", v.size, desc, 1)
    assert line["impl"] == "reference" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_bench_workload_is_the_generator_array():
    v, _ = bench._workload("plain_large", 0)
    assert np.array_equal(v, plain_large())
