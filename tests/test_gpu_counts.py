"""The executed-operation counters of the Miller-Rabin stages
(isprime_count_ops), checked exactly on an input whose schedule can be
worked out by hand, and against the oracle's canonical count on the
benchmark array.

Hand count for 64 copies of n = 2^61 - 1 (prime, s = 1, d = 2^60 - 1: 60 bits,
15 nibbles; no trial prime divides it):
* base 2, 4-bit windows with the estimated-quotient step: the first nibble
  is one step from 1, then 14 x (4 squarings + 1 step): 56 squarings and
  15 steps per value, no tail (s = 1).  Two full warps of 32 values (or one
  task of 64 values, two per thread): 112 squaring issues, 30 step issues,
  32 active lanes each.
* six bases: a queue of 64 is short, so the kernel spreads (survivor, base)
  pairs over threads: 384 pairs, 12 full warps, one base per lane.  Per warp:
  R^2 mod n (3 squarings), the base to Montgomery form (1 product), then
  4-bit windows: table 1 squaring + 13 products, 14 x (4 squarings + 1
  product): 60 squarings and 28 products; 3-bit windows (20 digits): table
  1 squaring + 5 products, 19 x (3 squarings + 1 product): 61 squarings and
  25 products.
"""
import numpy as np
import pytest

import oracle
from workloads import plain_large

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    with ipg.Context(0) as c:
        yield c


@pytest.mark.parametrize("ilp,win", [(1, 4), (2, 4), (1, 3), (2, 3)])
def test_counts_exact_on_a_hand_derived_input(ilp, win, ctx):
    ctx.set_tuning(base2_window=1, base2_ilp=ilp, rest_window=win, compact_min=33, td2_groups=0)
    v = np.full(64, 2**61 - 1, dtype=np.uint64)
    t = torch.from_numpy(v.view(np.int64)).to("cuda:0")
    c = ctx.count_ops(t)
    assert c["elements"] == 64
    assert c["base2_squarings"] == (112, 112 * 32)
    assert c["base2_steps"] == (30, 30 * 32)
    assert c["base2_products"] == (0, 0)
    sq, mul = (60, 28) if win == 4 else (61, 25)
    assert c["rest_squarings"] == (12 * sq, 12 * sq * 32)
    assert c["rest_products"] == (12 * mul, 12 * mul * 32)
    # the counting build gives the same answers
    assert ctx.isprime(t).cpu().numpy().tolist() == [1] * 64


def test_counts_bound_the_canonical_count_on_the_bench_array(ctx):
    """On 2^22 values of the benchmark array: the lanes that carried a value
    executed at least the canonical squarings of the binary schedule minus
    what the windows save (at most one squaring per value per base, the top
    digit's), and the warps paid at most a bounded padding over them."""
    ctx.set_tuning(base2_window=1, base2_ilp=1, rest_window=4, compact_min=33, td2_groups=0)
    v = plain_large(1 << 22, seed=1)
    t = torch.from_numpy(v.view(np.int64)).to("cuda:0")
    c = ctx.count_ops(t)
    w = oracle.work_counts(v, td_bound=53)
    b2_issue, b2_lanes = c["base2_squarings"]
    # every value's squarings are carried by an active lane: the windows do
    # bitlen(d) - 1 rounded down to whole nibbles, at most 3 fewer than binary
    assert b2_lanes >= w["base2_squarings"] - 3 * w["mr64_elements"]
    assert 32 * b2_issue >= b2_lanes
    # padding to the warp's largest nibble count and tail stays below 25%
    assert 32 * b2_issue <= 1.25 * (w["base2_squarings"] + 4 * w["mr64_elements"])
    r_issue, r_lanes = c["rest_squarings"]
    assert r_lanes >= w["rest_squarings"] - 6 * 3 * w["base2_passes"]
    assert 32 * r_issue <= 1.25 * (w["rest_squarings"] + 6 * 4 * w["base2_passes"])


def test_counts_follow_the_two_stage_schedule():
    """With the second trial stage (td2_groups 16: the primes 59..311 in the
    base-2 kernel) the base-2 squarings carried by active lanes follow the
    oracle's count at trial bound 311 (the windows do up to 3 fewer per value
    than the binary schedule), not the count at 53; the six-base
    kernel's work is that of the one-stage schedule, as no prime is removed."""
    ctx_tuning = dict(base2_window=1, base2_ilp=1, rest_window=3, compact_min=33, td2_groups=16)
    v = plain_large(1 << 22, seed=1)
    t = torch.from_numpy(v.view(np.int64)).to("cuda:0")
    with ipg.Context(0) as c:
        c.set_tuning(**ctx_tuning)
        got = c.count_ops(t)
    w311 = oracle.work_counts(v, td_bound=311)
    w53 = oracle.work_counts(v, td_bound=53)
    lanes = got["base2_squarings"][1]
    # (lanes also square the Montgomery 1 for leading zero digits below the
    # warp's largest digit count: a fraction of a percent here)
    assert w311["base2_squarings"] - 3 * w311["mr64_elements"] <= lanes <= 1.01 * w311["base2_squarings"]
    assert lanes < 0.8 * w53["base2_squarings"]
    assert w311["base2_passes"] == w53["base2_passes"]
    r_lanes = got["rest_squarings"][1]
    assert r_lanes >= w53["rest_squarings"] - 6 * 3 * w53["base2_passes"]
