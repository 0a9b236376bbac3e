"""GPU parity: the CUDA path against the CPU oracle, bit for bit.

Primality has exactly one right answer per element, so the bar is
bit-exact equality (tolerance 0).  Inputs come from the seeded generators in
`workloads`; expected values come only from the oracle (or from paper /
mathematical constants).  Every call goes through the C ABI (via the thin
ctypes binding).
"""
import numpy as np
import pytest

import oracle
from workloads import plain_small, plain_large, plain_mixed, mixed_doubles, bitlen_uniform

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _to_dev(vals):
    return torch.from_numpy(np.ascontiguousarray(vals, dtype=np.uint64).view(np.int64)).to(_dev())


def _gpu(vals, ctx=None):
    t = _to_dev(vals)
    out = (ctx.isprime(t) if ctx is not None else ipg.isprime(t))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _assert_same(vals, got, want):
    bad = np.flatnonzero(got != want)
    if bad.size:
        i = int(bad[0])
        raise AssertionError(f"{bad.size} mismatches; first at {i}: n={int(vals[i])} "
                             f"gpu={int(got[i])} oracle={int(want[i])}")


@pytest.fixture(scope="module")
def ctx_nosieve():
    _dev()
    with ipg.Context(0, sieve_limit=0) as c:
        yield c


@pytest.fixture(scope="module")
def ctx_small_sieve():
    _dev()
    with ipg.Context(0, sieve_limit=1 << 20) as c:
        yield c


# ------------------------------------------------------------------ workloads

def test_plain_small_full():
    v = plain_small()
    _assert_same(v, _gpu(v), oracle.isprime_u64(v))


def test_plain_large_2p20():
    v = plain_large(1 << 20)
    _assert_same(v, _gpu(v), oracle.isprime_u64(v))


def test_plain_large_full_size():
    """The benchmark's workload at its full size (2^24), every element."""
    v = plain_large()
    _assert_same(v, _gpu(v), oracle.isprime_u64(v))


def test_plain_mixed_2p22():
    v = plain_mixed(1 << 22)
    _assert_same(v, _gpu(v), oracle.isprime_u64(v))


def test_mixed_doubles():
    x = mixed_doubles(1 << 20)
    t = torch.from_numpy(x).to(_dev())
    inv = torch.zeros(1, dtype=torch.int64, device=_dev())
    out = ipg.isprime(t, invalid=inv)
    torch.cuda.synchronize()
    want, bad = oracle.isprime_f64(x)
    _assert_same(x.astype(np.uint64), out.cpu().numpy(), want)
    assert int(inv.item()) == bad == 0


def test_f64_domain_and_invalid_count(ctx_small_sieve):
    x = np.array([0.0, -0.0, 1.0, 2.0, 7.0, 9.0, 2.0**53, 2.0**53 - 111, float("nan"),
                  float("inf"), -float("inf"), -7.0, 2.5, 2.0**53 + 2, 1e300, 97.0, 3.0],
                 dtype=np.float64)
    old = ctx_small_sieve.tuning.small_max
    ctx_small_sieve.set_tuning(small_max=0)  # the queue path (classify_kernel<f64>)
    try:
        for k in (1, 2, 3, len(x)):  # ragged lengths through head/tail paths
            t = torch.from_numpy(x[:k].copy()).to(_dev())
            inv = torch.zeros(1, dtype=torch.int64, device=_dev())
            out = ctx_small_sieve.isprime(t, invalid=inv)
            torch.cuda.synchronize()
            want, bad = oracle.isprime_f64(x[:k])
            assert out.cpu().numpy().tolist() == want.tolist()
            assert int(inv.item()) == bad
    finally:
        ctx_small_sieve.set_tuning(small_max=old)


def _f64_call(ctx, x, stream=None, invalid=None):
    """isprime_f64_ctx through the C ABI; returns the output bytes."""
    import ctypes
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(_dev())
    out = torch.empty(t.numel(), dtype=torch.uint8, device=_dev())
    s = stream or torch.cuda.current_stream(_dev())
    st = ipg.lib().isprime_f64_ctx(ctx.handle, t.data_ptr(), out.data_ptr(), t.numel(),
                                   None if invalid is None else ctypes.c_void_p(invalid.data_ptr()),
                                   ctypes.c_void_p(s.cuda_stream))
    assert st == ipg.OK, st
    return t, out


@pytest.mark.parametrize("small_max", [0, 1 << 20])
def test_f64_sync_status_reports_edomain(small_max):
    """The EDOMAIN contract: invalid doubles (NaN, infinities, negatives,
    fractions, values above 2^53) are counted by the context itself even when
    the caller passes no counter, and isprime_f64_sync_status returns
    ISPRIME_EDOMAIN with that count, then resets it.  Calls on two streams
    are both counted.  Checked on the queue path (small_max 0) and on the
    one-launch path."""
    import ctypes
    L = ipg.lib()
    good = np.array([2.0, 3.0, 97.0, 2.0**53 - 111, 0.0], dtype=np.float64)
    bad = np.array([float("nan"), -1.0, 2.5, 2.0**53 + 2, float("inf"), 1e300, 7.0],
                   dtype=np.float64)
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        c.set_tuning(small_max=small_max)
        cnt = ctypes.c_ulonglong(99)
        assert L.isprime_f64_sync_status(c.handle, ctypes.byref(cnt)) == ipg.OK
        assert cnt.value == 0
        _, out = _f64_call(c, good)  # no invalid element: still OK
        assert L.isprime_f64_sync_status(c.handle, ctypes.byref(cnt)) == ipg.OK and cnt.value == 0
        assert out.cpu().numpy().tolist() == oracle.isprime_f64(good)[0].tolist()
        s2 = torch.cuda.Stream(_dev())
        keep = [_f64_call(c, bad), _f64_call(c, np.concatenate([bad, good]), stream=s2)]
        want_bad = oracle.isprime_f64(bad)[1]
        assert want_bad == 6
        assert L.isprime_f64_sync_status(c.handle, ctypes.byref(cnt)) == ipg.EDOMAIN
        assert cnt.value == 2 * want_bad
        assert b"2^53" in L.isprime_last_error()
        # the status call reset the count
        assert L.isprime_f64_sync_status(c.handle, None) == ipg.OK
        # a caller's counter and the context's count agree
        inv = torch.zeros(1, dtype=torch.int64, device=_dev())
        keep.append(_f64_call(c, bad, invalid=inv))
        assert c.f64_status() == want_bad
        torch.cuda.synchronize()
        assert int(inv.item()) == want_bad
        for (t, out), x in zip(keep, [bad, np.concatenate([bad, good]), bad]):
            assert out.cpu().numpy().tolist() == oracle.isprime_f64(x)[0].tolist()
        # the u64 path never counts
        _gpu(np.array([1, 2, 3], dtype=np.uint64), c)
        assert c.f64_status() == 0
    assert L.isprime_f64_sync_status(None, None) == ipg.EINVAL


# ------------------------------------------------------------------ edge cases

SPECIAL = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 25, 49, 121, 169, 251, 253, 257, 65521, 65537,
           561, 1105, 1729, 2047, 3277, 4033, 4681, 8321, 3215031751, 2152302898747,
           3474749660383, 341550071728321, 3825123056546413051,
           2**31 - 1, 2**32 - 5, 2**32 - 1, 2**32, 2**32 + 1, 2**32 + 15, 2**48 - 59,
           2**52 - 47, 2**53 - 111, 2**61 - 1, 2**62 - 57, 2**63 - 25, 2**63, 2**63 + 1,
           2**64 - 59, 2**64 - 57, 2**64 - 3, 2**64 - 1, 4759123141, 1122004669633]


@pytest.mark.parametrize("which", ["default", "nosieve", "smallsieve"])
def test_special_values(which, ctx_nosieve, ctx_small_sieve):
    ctx = {"default": None, "nosieve": ctx_nosieve, "smallsieve": ctx_small_sieve}[which]
    v = np.array(SPECIAL, dtype=np.uint64)
    want = oracle.isprime_u64(v)
    _assert_same(v, _gpu(v, ctx), want)  # short array: the one-warp-per-element path
    if ctx is not None:                  # and the queue path of the same context
        old = ctx.tuning.small_max
        ctx.set_tuning(small_max=0)
        try:
            _assert_same(v, _gpu(v, ctx), want)
        finally:
            ctx.set_tuning(small_max=old)


def test_empty_input():
    t = torch.empty(0, dtype=torch.int64, device=_dev())
    assert ipg.isprime(t).numel() == 0


@pytest.mark.parametrize("small_max", [0, None])
def test_ragged_lengths_and_offsets(small_max, ctx_small_sieve):
    """Short arrays on the queue path (small_max = 0: head element, pair
    stores, odd tails) and on the one-launch warp path (the default)."""
    base = plain_mixed(4096, seed=9)
    big = _to_dev(base)
    want_all = oracle.isprime_u64(base)
    old = ctx_small_sieve.tuning.small_max
    if small_max is not None:
        ctx_small_sieve.set_tuning(small_max=small_max)
    try:
        for off in (0, 1, 2, 3):
            for n in list(range(1, 70)) + [127, 128, 129, 1023, 1025, 4093]:
                t = big[off:off + n]          # misaligned by 8 bytes for odd off
                out = torch.zeros(n + 3, dtype=torch.uint8, device=_dev())[1:n + 1]  # odd output address
                ctx_small_sieve.isprime(t, out=out)
                torch.cuda.synchronize()
                assert out.cpu().numpy().tolist() == want_all[off:off + n].tolist(), (off, n)
    finally:
        ctx_small_sieve.set_tuning(small_max=old)


def test_no_sieve_and_small_sieve_contexts(ctx_nosieve, ctx_small_sieve):
    v = np.concatenate([plain_mixed(1 << 20, seed=11), np.arange(0, 70000, dtype=np.uint64)])
    want = oracle.isprime_u64(v)
    _assert_same(v, _gpu(v, ctx_nosieve), want)
    _assert_same(v, _gpu(v, ctx_small_sieve), want)


def test_windows_at_boundaries():
    """Consecutive integers around 2^20, 2^24, 2^32 and below 2^64."""
    for lo in (1 << 20, (1 << 24) - 5000, (1 << 32) - 50000, (1 << 64) - 100000):
        v = np.uint64(lo) + np.arange(100000, dtype=np.uint64)  # last window ends at 2^64 - 1
        _assert_same(v, _gpu(v), oracle.isprime_u64(v))


def test_strong_pseudoprimes_and_carmichaels(ctx_nosieve):
    import numtheory as nt
    N = 2_000_000
    comp = ~nt.simple_sieve(N)
    spsp = [n for n in range(9, N, 2) if comp[n] and nt.strong_base2(n)]
    cars = []
    for k in range(1, 1 << 20):
        a, b, c = 6 * k + 1, 12 * k + 1, 18 * k + 1
        if a * b * c >= 1 << 64:
            break
        if nt.trial_is_prime(a) and nt.trial_is_prime(b) and nt.trial_is_prime(c):
            cars.append(a * b * c)
    v = np.array(spsp + cars, dtype=np.uint64)
    assert not _gpu(v).any()
    assert not _gpu(v, ctx_nosieve).any()


def test_tuning_does_not_change_results():
    v = np.concatenate([plain_large(1 << 18, seed=21), plain_mixed(1 << 18, seed=22)])
    want = oracle.isprime_u64(v)
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        for kw in [dict(td_primes=0), dict(td_primes=1), dict(td_primes=53),
                   dict(classify_block=64, mr_block=32, blocks_per_sm=1),
                   dict(classify_block=1024, mr_block=256, blocks_per_sm=16),
                   dict(chunk_log2=16), dict(mont_impl=1), dict(mont_impl=2),
                   dict(mont_impl=3), dict(mont_impl=4), dict(mont_impl=5),
                   dict(mont_impl_base2=0), dict(mont_impl_base2=1), dict(mont_impl_base2=2),
                   dict(mont_impl_base2=3), dict(mont_impl_base2=4), dict(mont_impl_base2=5),
                   dict(td_primes=7), dict(td_primes=11), dict(td_primes=23), dict(td_primes=31),
                   dict(td_primes=40), dict(base2_window=0), dict(base2_window=4, mont_impl_base2=0),
                   dict(base2_window=4), dict(base2_window=1, mont_impl_base2=0),
                   dict(base2_window=4, compact_min=8), dict(base2_window=1, compact_min=8),
                   dict(base2_window=1, compact_min=4, rest_test=1),
                   dict(rest_test=1), dict(rest_test=1, mont_impl=5), dict(rest_test=0),
                   dict(mont_impl=0, td_primes=15), dict(mont_impl=6), dict(mont_impl_base2=6),
                   dict(mont_impl=6, mont_impl_base2=6, base2_window=0),
                   dict(mont_impl=6, rest_test=1), dict(mont_impl_base2=6, compact_min=8),
                   dict(mont_impl=7), dict(mont_impl=8), dict(mont_impl_base2=7),
                   dict(mont_impl_base2=8), dict(mont_impl=7, mont_impl_base2=8, base2_window=0),
                   dict(mont_impl=8, rest_test=1), dict(mont_impl_base2=7, base2_window=4),
                   dict(mont_impl=7, compact_min=8), dict(mont_impl=9), dict(mont_impl_base2=9),
                   dict(mont_impl=9, mont_impl_base2=9, base2_window=0),
                   dict(mont_impl=9, rest_window=4), dict(mont_impl_base2=9, base2_window=4),
                   dict(pdl=1), dict(pdl=1, sieve_cutover_log2=20), dict(pdl=1, base2_window=0),
                   dict(pdl=1, rest_test=1), dict(pdl=1, chunk_log2=16), dict(pdl=0),
                   dict(compact_min=0), dict(compact_min=1), dict(compact_min=16),
                   dict(compact_min=1, base2_window=4), dict(compact_min=0, rest_test=1),
                   dict(compact_min=1, base2_window=0), dict(compact_min=1, chunk_log2=16),
                   dict(compact_min=0, base2_window=1, chunk_log2=24),
                   dict(compact_min=4, rest_test=1), dict(compact_min=8, mont_impl_base2=5),
                   dict(compact_min=2, base2_window=0), dict(compact_min=33),
                   dict(sieve_cutover_log2=0), dict(sieve_cutover_log2=20),
                   dict(sieve_cutover_log2=23, td_primes=0), dict(sieve_cutover_log2=32),
                   dict(inplace_max_log2=20, chunk_log2=24), dict(inplace_max_log2=16, chunk_log2=16),
                   dict(inplace_max_log2=20, rest_test=1), dict(inplace_max_log2=20, base2_window=0),
                   dict(inplace_max_log2=0, base2_window=2, rest_test=0),
                   dict(base2_window=2, compact_min=8), dict(base2_window=2, compact_min=33,
                                                             base2_ilp=2),
                   dict(base2_window=2, mont_impl_base2=6), dict(base2_window=2, td2_groups=0)]:
            c.set_tuning(**kw)
            _assert_same(v, _gpu(v, c), want)


def test_sieve_counts():
    assert ipg.Context.default(0).sieve_count() == 203280221  # pi(2^32)
    with ipg.Context(0, sieve_limit=1 << 20) as c:
        assert c.sieve_count() == 82025                           # pi(2^20)
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        assert c.sieve_count() == 1077871                         # pi(2^24)


def test_mr32_exhaustive_against_sieve(ctx_small_sieve):
    """Every odd n in [2^20, 2^32): 32-bit Miller-Rabin with bases {2,7,61}
    (context with S = 2^20) equals the sieve lookup of the default context
    (S = 2^32), whose bitmap is pinned by pi(2^32)."""
    dev = _dev()
    default = ipg.Context.default(0)
    step = 1 << 27
    lo = 1 << 20
    total = 0
    while lo < (1 << 32):
        hi = min(lo + 2 * step, 1 << 32)
        t = torch.arange(lo + 1, hi, 2, dtype=torch.int64, device=dev)
        a = ctx_small_sieve.isprime(t)
        b = default.isprime(t)
        torch.cuda.synchronize()
        if not torch.equal(a, b):
            i = int(torch.nonzero(a != b)[0])
            raise AssertionError(f"MR32 vs sieve differ at n={int(t[i])}")
        total += int(a.sum())
        lo = hi
    # odd primes in [2^20, 2^32) = pi(2^32) - pi(2^20)
    assert total == 203280221 - 82025


def test_host_path_matches_device_path():
    v = plain_mixed(300_001, seed=31)
    c = ipg.Context.default(0)
    got = c.isprime_host(v)
    _assert_same(v, got, oracle.isprime_u64(v))


@pytest.mark.parametrize("n,host_log2", [((1 << 20) + 4097, 16), ((1 << 21) + 3, 18),
                                         (5 * (1 << 18) + 77, 17), ((1 << 16) + 1, 16)])
def test_host_path_many_chunks_reuse_every_staging_slot(n, host_log2):
    """isprime_u64_host with chunks of at most 2^host_chunk_log2 values: the
    ramp-up chunks, then equal chunks, the four staging slots each reused
    several times (a slot's refill waits for the chunk four back to be
    computed and copied out) and the two compute streams alternating; two
    calls in a row with different inputs."""
    v1 = plain_mixed(n, seed=43)
    v2 = plain_large(n, seed=44)
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        c.set_tuning(host_chunk_log2=host_log2, small_max=0)
        _assert_same(v1, c.isprime_host(v1), oracle.isprime_u64(v1))
        _assert_same(v2, c.isprime_host(v2), oracle.isprime_u64(v2))
        with pytest.raises(ipg.IsPrimeError):
            c.set_tuning(host_chunk_log2=15)
        with pytest.raises(ipg.IsPrimeError):
            c.set_tuning(host_chunk_log2=25)


def test_two_streams_share_one_context():
    v1 = plain_large(1 << 18, seed=41)
    v2 = plain_mixed(1 << 18, seed=42)
    t1, t2 = _to_dev(v1), _to_dev(v2)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        o1 = ipg.isprime(t1)
    with torch.cuda.stream(s2):
        o2 = ipg.isprime(t2)
    torch.cuda.synchronize()
    _assert_same(v1, o1.cpu().numpy(), oracle.isprime_u64(v1))
    _assert_same(v2, o2.cpu().numpy(), oracle.isprime_u64(v2))


def test_timing_records_every_kernel():
    c = ipg.Context.default(0)
    c.timing_reset()
    c.timing(True)
    v = _to_dev(plain_large(1 << 20, seed=51))
    c.isprime(v)
    torch.cuda.synchronize()
    rec = c.timing_read()
    c.timing(False)
    assert rec["classify_u64"][1] == 1 and rec["mr64_base2"][1] == 1 and rec["mr64_rest"][1] == 1
    assert all(ms > 0 for ms, n in rec.values() if n)


def test_int_rates_probe():
    r = ipg.int_rates(0)
    assert r["mad_lo_u32"] > 1e12 and r["mont_mul_128"] > 1e10 and r["sm_clock_mhz"] > 100


# ------------------------------------------------------------------ batched

def test_batched_matches_oracle_on_ragged_batch():
    from workloads import batched_arrays
    vals, offs = batched_arrays(n_arrays=300, max_size=1 << 14, seed=61)
    sizes = np.diff(offs)
    # add edge cases: empty arrays, single elements, special values
    extra = [np.array([], dtype=np.uint64), np.array([2**64 - 59], dtype=np.uint64),
             np.array(SPECIAL, dtype=np.uint64), np.array([], dtype=np.uint64)]
    arrays = [vals[offs[i]:offs[i + 1]] for i in range(len(sizes))] + extra
    c = ipg.Context.default(0)
    tens = [_to_dev(a) for a in arrays]
    outs = c.isprime_batched(tens)
    torch.cuda.synchronize()
    for a, o in zip(arrays, outs):
        _assert_same(a, o.cpu().numpy(), oracle.isprime_u64(a))


def test_batched_rejects_tuning_beyond_shared_memory():
    with pytest.raises(ipg.IsPrimeError):
        ipg.Context.default(0).set_tuning(batch_block=256, batch_tile_log2=14)


@pytest.mark.parametrize("kw", [dict(), dict(batch_block=64, batch_tile_log2=8),
                                dict(batch_block=256, batch_tile_log2=13),
                                dict(batch_block=64, batch_tile_log2=13),
                                dict(td_primes=23), dict(td_primes=5),
                                dict(batch_blocks_per_sm=1), dict(sieve_cutover_log2=16),
                                dict(sieve_cutover_log2=0, td_primes=0)])
def test_batched_tuning_and_small_sieve(kw):
    from workloads import batched_arrays
    vals, offs = batched_arrays(n_arrays=64, max_size=1 << 15, seed=62)
    arrays = [vals[offs[i]:offs[i + 1]] for i in range(64)]
    with ipg.Context(0, sieve_limit=1 << 20) as c:
        c.set_tuning(**kw)
        for _ in range(2):  # second call replays the recorded graph
            outs = c.isprime_batched([_to_dev(a) for a in arrays])
            torch.cuda.synchronize()
            for a, o in zip(arrays, outs):
                _assert_same(a, o.cpu().numpy(), oracle.isprime_u64(a))


@pytest.mark.parametrize("n_arrays", [1, 2, 31, 33, 700, 1500])
def test_batched_short_batch_takes_the_warp_form(n_arrays):
    """A batch of at most small_max elements runs as one warp-per-element
    launch (element prefix sums, 32-way array search); results equal the
    persistent kernel's and the oracle's, empty arrays included."""
    rng = np.random.default_rng(n_arrays)
    sizes = rng.integers(0, 12, size=n_arrays)
    sizes[::5] = 0
    vals = np.concatenate([np.array(SPECIAL * 3, dtype=np.uint64), plain_mixed(20000, seed=64)])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    arrays = [vals[offs[i]:offs[i + 1]] for i in range(n_arrays)]
    with ipg.Context(0) as c:
        for small_max in (1 << 20, 0):
            c.set_tuning(small_max=small_max)
            c.timing_reset()
            c.timing(True)
            outs = c.isprime_batched([_to_dev(a) for a in arrays])
            torch.cuda.synchronize()
            rec = c.timing_read()
            c.timing(False)
            for a, o in zip(arrays, outs):
                _assert_same(a, o.cpu().numpy(), oracle.isprime_u64(a))
            if sizes.sum():
                assert (rec["small"][1], rec["batched"][1]) == ((1, 0) if small_max else (0, 1))


def test_batched_and_plain_calls_match_oracle():
    """The same arrays (empty, one value, ragged) through one batched launch
    and through one plain call each: both equal the oracle."""
    vals = plain_mixed(1 << 18, seed=63)
    parts = np.split(vals, [1, 10, 1000, 50000, 50001])
    c = ipg.Context.default(0)
    outs = c.isprime_batched([_to_dev(p) for p in parts])
    plain = [_gpu(p, c) if p.size else np.zeros(0, np.uint8) for p in parts]
    torch.cuda.synchronize()
    for o, p, v in zip(outs, plain, parts):
        want = oracle.isprime_u64(v)
        _assert_same(v, o.cpu().numpy(), want)
        _assert_same(v, p, want)


# ------------------------------------------------------------------ autotuner

def test_autotune_keeps_results_exact_and_caches(tmp_path):
    v = np.concatenate([plain_large(1 << 17, seed=81), plain_mixed(1 << 17, seed=82)])
    want = oracle.isprime_u64(v)
    cache = str(tmp_path / "tune.txt")
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        t1 = c.autotune(_to_dev(v), mode="plain", cache_path=cache)
        _assert_same(v, _gpu(v, c), want)
        tb = c.autotune(_to_dev(v), mode="batched", cache_path=cache)
        outs = c.isprime_batched([_to_dev(v[:1000]), _to_dev(v[1000:])])
        torch.cuda.synchronize()
        _assert_same(v, np.concatenate([o.cpu().numpy() for o in outs]), want)
    lines = open(cache).read().splitlines()
    assert len(lines) == 2 and all("td_primes=" in l for l in lines)
    with ipg.Context(0, sieve_limit=1 << 24) as c2:  # a cache hit installs the same tuning
        assert c2.autotune(_to_dev(v), mode="plain", cache_path=cache) == t1
        assert c2.autotune(_to_dev(v), mode="batched", cache_path=cache) == tb


# ------------------------------------------------------------------ range form

def _range(ctx, lo, count):
    out = ctx.isprime_range(lo, count)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("lo,count", [(0, 10**6), (1, 999_999), (7, 1), (2, 3),
                                      ((1 << 32) - 100_000, 200_000),
                                      ((1 << 40) + 1, (1 << 21) + 3),
                                      ((1 << 64) - (1 << 20), 1 << 20),
                                      ((1 << 64) - 5, 5)])
def test_range_matches_oracle(lo, count, ctx_nosieve, ctx_small_sieve):
    vals = np.uint64(lo) + np.arange(count, dtype=np.uint64)
    want = oracle.isprime_u64(vals)
    for ctx in (ipg.Context.default(0), ctx_nosieve, ctx_small_sieve):
        _assert_same(vals, _range(ctx, lo, count), want)


def test_range_unix_seconds_2021_and_pi_1e8():
    """Table 5's window (the Unix seconds of 2021) and Table 3's 1:10^8."""
    lo, count = 1609477200, 3600 * 24 * 365 + 1
    vals = np.uint64(lo) + np.arange(count, dtype=np.uint64)
    ctx = ipg.Context.default(0)
    _assert_same(vals, _range(ctx, lo, count), oracle.isprime_u64(vals))
    out = ctx.isprime_range(1, 10**8)
    assert int(out.sum().item()) == 5761455  # pi(10^8)
    with ipg.Context(0, sieve_limit=0) as c0:  # the sieve path gives the same count
        assert int(c0.isprime_range(1, 10**8).sum().item()) == 5761455


def test_range_misaligned_output_and_argument_checks():
    ctx = ipg.Context.default(0)
    buf = torch.zeros(1003, dtype=torch.uint8, device="cuda")
    ctx.isprime_range(999_983, 1000, out=buf[3:])   # output starts at an odd address
    torch.cuda.synchronize()
    vals = np.uint64(999_983) + np.arange(1000, dtype=np.uint64)
    assert buf[3:].cpu().numpy().tolist() == oracle.isprime_u64(vals).tolist()
    with pytest.raises(ipg.IsPrimeError):
        ctx.isprime_range((1 << 64) - 3, 4)          # lo + count > 2^64


def test_range_expand_ends_at_the_sieve_limit():
    """Windows that end exactly at S (the last bitmap word) and cross it."""
    with ipg.Context(0, sieve_limit=1 << 20) as c:
        for lo, count in [((1 << 20) - 4096, 4096), ((1 << 20) - 17, 17), ((1 << 20) - 33, 100),
                          ((1 << 20) - 16, 16)]:
            vals = np.uint64(lo) + np.arange(count, dtype=np.uint64)
            _assert_same(vals, _range(c, lo, count), oracle.isprime_u64(vals))


# ------------------------------------------------------------------ Baillie-PSW option

@pytest.fixture(scope="module")
def ctx_bpsw():
    _dev()
    with ipg.Context(0) as c:
        c.set_tuning(rest_test=1)
        yield c


def test_bpsw_full_bench_array_and_mixed(ctx_bpsw):
    for v in (plain_large(), plain_mixed(1 << 22, seed=101), np.array(SPECIAL, dtype=np.uint64)):
        _assert_same(v, _gpu(v, ctx_bpsw), oracle.isprime_u64(v))


def test_bpsw_rejects_base2_strong_pseudoprimes(ctx_bpsw):
    """Composites that pass the base-2 stage: the Lucas stage must reject them."""
    import random
    import numtheory as nt
    rng = random.Random(103)
    spsp = []
    while len(spsp) < 40:  # p (2p - 1) with both prime, near 2^63, that pass base 2
        p = rng.randrange(2**31, 3_000_000_000) | 1
        q = 2 * p - 1
        if nt.trial_is_prime(p) and nt.trial_is_prime(q) and nt.strong_base2(p * q):
            spsp.append(p * q)
    N = 2_000_000
    comp = ~nt.simple_sieve(N)
    small = [n for n in range(9, N, 2) if comp[n] and nt.strong_base2(n)]
    v = np.array(spsp + small, dtype=np.uint64)
    assert not _gpu(v, ctx_bpsw).any()
    with ipg.Context(0, sieve_limit=0) as c0:  # small ones through MR32 / Lucas, no sieve
        c0.set_tuning(rest_test=1)
        assert not _gpu(v, c0).any()


def _spsp_near_2p63(count, seed):
    import random
    import numtheory as nt
    rng = random.Random(seed)
    out = []
    while len(out) < count:  # p (2p - 1) with both prime, near 2^63, that pass base 2
        p = rng.randrange(2**31, 3_000_000_000) | 1
        q = 2 * p - 1
        if nt.trial_is_prime(p) and nt.trial_is_prime(q) and nt.strong_base2(p * q):
            out.append(p * q)
    return out


@pytest.mark.parametrize("window", [0, 1, 4])
def test_base2_schedules_on_every_bit_size(window):
    """The three base-2 schedules (binary with doublings; 4-bit windows whose
    step x 2^w mod n uses an estimated quotient; 4-bit windows over a table)
    on the queue path: random odd values of every size from 33 to 64 bits
    (normalising shifts 31 down to 0), the primes among them and their odd
    neighbours, the odd values just above 2^32 and just below 2^64, and
    base-2 strong pseudoprimes p (2p - 1) near 2^63, which must reach the
    other bases."""
    rng = np.random.default_rng(131)
    cand = np.concatenate([rng.integers(1 << (b - 1), (1 << b) - 1, size=2000, dtype=np.uint64,
                                        endpoint=True) | np.uint64(1) for b in range(33, 65)])
    primes = cand[oracle.isprime_u64(cand).astype(bool)]
    near = primes[primes < np.uint64(2**64 - 2)] + np.uint64(2)
    edges = np.array(list(range(2**32 + 1, 2**32 + 400, 2)) + list(range(2**64 - 399, 2**64, 2))
                     + _spsp_near_2p63(16, seed=131), dtype=np.uint64)
    v = np.concatenate([cand, near, primes - np.uint64(2), edges])
    want = oracle.isprime_u64(v)
    assert want.sum() > 2000
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        c.set_tuning(base2_window=window, small_max=0)
        _assert_same(v, _gpu(v, c), want)


@pytest.fixture(scope="module")
def ctx_mr128():
    with ipg.Context(0) as c:
        c.set_tuning(mr_block=128)
        yield c


@pytest.mark.parametrize("log2n", [20, 21, 22])
def test_rest_queue_spread_factors(log2n, ctx_mr128):
    """2^20, 2^21 and 2^22 large values give base-2 survivor queues of about
    36K, 73K and 145K entries: with 128-thread blocks the rest kernel's grid of
    2432 blocks (311K threads) takes them with 6, 3 and 2 threads per
    survivor; with the default 256-thread blocks, 6, 6 and 3."""
    v = plain_large(1 << log2n, seed=110 + log2n)
    want = oracle.isprime_u64(v)
    _assert_same(v, _gpu(v, ctx_mr128), want)
    _assert_same(v, _gpu(v), want)


@pytest.mark.parametrize("n", [1, 7, 64, 1000, 5000, 40000])
def test_short_queues_spread_over_bases(n, ctx_small_sieve):
    """Chunks short enough for one (survivor, base) pair per thread: primes near
    2^64 (every base passes) mixed with base-2 strong pseudoprimes (a later base
    fails) and random large values, on the queue path (small_max = 0)."""
    from workloads import load_pool
    rng = np.random.default_rng(n)
    primes = load_pool("primes_near_2p64.txt")
    spsp = np.array(_spsp_near_2p63(12, seed=n), dtype=np.uint64)
    v = np.concatenate([primes[rng.integers(0, primes.size, n)], spsp, plain_large(n, seed=n + 5)])
    rng.shuffle(v)
    v = v[:max(n, 1)] if n < spsp.size else v
    want = oracle.isprime_u64(v)
    old = ctx_small_sieve.tuning.small_max
    ctx_small_sieve.set_tuning(small_max=0)
    try:
        _assert_same(v, _gpu(v, ctx_small_sieve), want)
    finally:
        ctx_small_sieve.set_tuning(small_max=old)


def test_bpsw_batched(ctx_bpsw):
    from workloads import batched_arrays
    vals, offs = batched_arrays(n_arrays=64, max_size=1 << 15, seed=104)
    arrays = [vals[offs[i]:offs[i + 1]] for i in range(64)]
    outs = ctx_bpsw.isprime_batched([_to_dev(a) for a in arrays])
    torch.cuda.synchronize()
    for a, o in zip(arrays, outs):
        _assert_same(a, o.cpu().numpy(), oracle.isprime_u64(a))
