"""The per-call path choice (window path) against the CPU oracle.

With window_ratio16 > 0, a uint64 call of at least 2^16 values whose values
fill a narrow window [min, max] above the resident sieve limit is classified
by sieving that window (the range kernels) and gathering; otherwise the queue
path runs.  Both arms must equal the oracle bit for bit; the context's
window_calls counter shows which arm ran.
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
    with ipg.Context(0, sieve_limit=1 << 32) as c:
        yield c


def _dense(lo, w, n, seed):
    """n values drawn from [lo, lo + w) (repeats allowed), every integer of a
    short run at both ends included so that min = lo and max = lo + w - 1."""
    rng = np.random.default_rng(seed)
    v = (np.uint64(lo) + rng.integers(0, w, size=n, dtype=np.uint64)).astype(np.uint64)
    v[:8] = np.array([lo + k for k in range(8)], dtype=np.uint64)
    v[-8:] = np.array([lo + w - 8 + k for k in range(8)], dtype=np.uint64)
    return v


def _run(ctx, v):
    t = torch.from_numpy(v.view(np.int64)).to("cuda:0")
    before = ctx.stats()["window_calls"]
    out = ctx.isprime(t)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ctx.stats()["window_calls"] - before


def _same(v, got, want, what):
    bad = np.flatnonzero(got != want)
    assert not bad.size, (f"{what}: {bad.size} mismatches; first n={int(v[bad[0]])} "
                          f"gpu={int(got[bad[0]])} oracle={int(want[bad[0]])}")


@pytest.mark.parametrize("lo,w,n", [
    (1 << 32, 1 << 20, 1 << 20),              # at the sieve limit
    ((1 << 32) - 1000, 1 << 18, 1 << 18),     # straddling the sieve limit
    (1 << 40, 3 * (1 << 17) + 7, 1 << 19),    # ragged window, repeats
    (2**49 + 12345, 1 << 19, 1 << 17),        # density 1/4
    (1 << 63, 1 << 20, 1 << 20),
    (2**64 - (1 << 20), 1 << 20, 1 << 20),    # ends at 2^64 - 1
])
def test_window_path_matches_oracle(lo, w, n, ctx):
    v = _dense(lo, w, n, seed=lo % 1000 + w)
    want = oracle.isprime_u64(v)
    ctx.set_tuning(window_ratio16=4096, small_max=0)
    try:
        got, taken = _run(ctx, v)
        _same(v, got, want, f"window lo={lo} w={w}")
        assert taken == 1
        ctx.set_tuning(window_ratio16=0)
        got, taken = _run(ctx, v)
        _same(v, got, want, f"queue lo={lo} w={w}")
        assert taken == 0
    finally:
        ctx.set_tuning(window_ratio16=0)


def test_rule_declines_sparse_low_and_short_arrays(ctx):
    ctx.set_tuning(window_ratio16=4096, small_max=0)
    try:
        v = plain_large(1 << 18, seed=5)               # sparse: W ~ 2^64
        got, taken = _run(ctx, v)
        _same(v, got, oracle.isprime_u64(v), "sparse")
        assert taken == 0
        v = _dense(10**9, 1 << 18, 1 << 18, seed=6)    # below the sieve limit: bit lookups
        got, taken = _run(ctx, v)
        _same(v, got, oracle.isprime_u64(v), "below S")
        assert taken == 0
        v = _dense(1 << 40, 1000, (1 << 16) - 1, seed=7)  # fewer than 2^16 values
        got, taken = _run(ctx, v)
        _same(v, got, oracle.isprime_u64(v), "short")
        assert taken == 0
        v = _dense(1 << 40, 1 << 25, 1 << 16, seed=8)  # 16 W > 4096 n: too sparse for the rule
        got, taken = _run(ctx, v)
        _same(v, got, oracle.isprime_u64(v), "ratio")
        assert taken == 0
    finally:
        ctx.set_tuning(window_ratio16=0)


def test_autotuner_fits_and_installs_the_crossover():
    """The autotuner installs its fitted crossover exactly when the sample
    itself is a window the fitted rule takes (whether the window path wins at
    a given density is this GPU's measurement, tabulated by the benchmark);
    a sparse sample keeps the path off.  Results stay exact either way."""
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        n, w = 1 << 22, 1 << 19  # density 8: every window integer about eight times
        v = _dense(1 << 44, w, n, seed=9)
        t = torch.from_numpy(v.view(np.int64)).to("cuda:0")
        tuned = c.autotune(t)
        r16 = tuned["window_ratio16"]
        assert r16 == 0 or 16 * w <= n * r16
        got, taken = _run(c, v)
        _same(v, got, oracle.isprime_u64(v), "tuned window")
        assert taken == (1 if r16 else 0)
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        v = plain_large(1 << 18, seed=10)
        tuned = c.autotune(torch.from_numpy(v.view(np.int64)).to("cuda:0"))
        assert tuned["window_ratio16"] == 0
