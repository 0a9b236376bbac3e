"""GPU parity of the kernel variants selected by tuning: folded trial
division (td_fold), the base-2 queue split by s (base2_split), two survivors
per thread in the base-2 kernel (base2_ilp) and 3-bit windows in the
six-base kernel (rest_window).

None of them may change a result, so every combination is compared with the
CPU oracle bit for bit, on inputs that reach every branch they touch: values
of every bit size from 33 to 64 (s = 1 and s >= 2, all fold residues),
primes and their neighbours, the odd values just above 2^32 and just below
2^64, multiples of every trial prime near 2^64, base-2 strong pseudoprimes
near 2^63 (they must reach the six-base kernel), ragged lengths, a
misaligned input pointer, several chunks per call, and the host-buffer path.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import numtheory as nt
from workloads import plain_large, plain_mixed
from workloads.generators import load_pool

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402

TRIAL_PRIMES = [3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53]


def _spsp_near_2p63(count, seed):
    rng = random.Random(seed)
    out = []
    while len(out) < count:  # p (2p - 1) with both prime, near 2^63, that pass base 2
        p = rng.randrange(2**31, 3_000_000_000) | 1
        q = 2 * p - 1
        if nt.trial_is_prime(p) and nt.trial_is_prime(q) and nt.strong_base2(p * q):
            out.append(p * q)
    return out


def _inputs():
    rng = np.random.default_rng(2024)
    cand = np.concatenate([rng.integers(1 << (b - 1), (1 << b) - 1, size=1200, dtype=np.uint64,
                                        endpoint=True) | np.uint64(1) for b in range(33, 65)])
    primes = cand[oracle.isprime_u64(cand).astype(bool)]
    near = primes[primes < np.uint64(2**64 - 2)] + np.uint64(2)
    # p * k near 2^64 and just above 2^32 for every trial prime: each fold must see them
    mult = []
    for p in TRIAL_PRIMES:
        top = (2**64 - 1) // p
        mult += [p * (top - j) for j in range(40)]
        low = (2**32) // p + 1
        mult += [p * (low + j) for j in range(40)]
        mult += [p * p * (((2**61) // (p * p)) + j) for j in range(10)]
    edges = (list(range(2**32 + 1, 2**32 + 300, 2)) + list(range(2**64 - 299, 2**64, 2))
             + _spsp_near_2p63(24, seed=7) + [2**61 - 1, 2**64 - 59, 3215031751, 4759123141])
    v = np.concatenate([cand, near, np.array(mult + edges, dtype=np.uint64),
                        plain_large(20_000, seed=91), plain_mixed(20_000, seed=92)])
    rng.shuffle(v)
    return v


@pytest.fixture(scope="module")
def data():
    v = _inputs()
    return v, oracle.isprime_u64(v)


@pytest.fixture(scope="module")
def ctx():
    with ipg.Context(0, sieve_limit=1 << 24) as c:
        yield c


def _run(c, v):
    t = torch.from_numpy(np.ascontiguousarray(v).view(np.int64)).to("cuda:0")
    out = c.isprime(t)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _same(v, got, want, what):
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (f"{what}: {bad.size} mismatches; first n={int(v[bad[0]])} "
                           f"gpu={int(got[bad[0]])} oracle={int(want[bad[0]])}")


COMBOS = list(itertools.product([0, 1, 2, 3], [0, 1], [1, 2], [3, 4]))


@pytest.mark.parametrize("fold,split,ilp,win", COMBOS)
def test_variant_matches_oracle(fold, split, ilp, win, data, ctx):
    v, want = data
    ctx.set_tuning(td_fold=fold, base2_split=split, base2_ilp=ilp, rest_window=win, small_max=0,
                   td_primes=15, chunk_log2=24, mont_impl=6, mont_impl_base2=6, base2_window=1,
                   compact_min=33)
    _same(v, _run(ctx, v), want, f"fold={fold} split={split} ilp={ilp} win={win}")


@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 63, 65, 1023, 4097, 70001])
def test_variants_on_ragged_and_misaligned(n, data, ctx):
    """Odd lengths, lengths around a warp task (32 and 64 survivors), and an
    input that starts 8 bytes past a 16-byte boundary."""
    v, want = data
    ctx.set_tuning(td_fold=2, base2_split=1, base2_ilp=2, rest_window=3, small_max=0,
                   chunk_log2=24)
    _same(v[:n], _run(ctx, v[:n]), want[:n], f"n={n}")
    t = torch.from_numpy(np.ascontiguousarray(v[:n + 1]).view(np.int64)).to("cuda:0")
    out = ctx.isprime(t[1:])
    torch.cuda.synchronize()
    _same(v[1:n + 1], out.cpu().numpy(), want[1:n + 1], f"misaligned n={n}")


def test_variants_over_several_chunks(data, ctx):
    """chunk_log2 = 16: the array runs as several chunks on one queue set, so
    both q64 regions are refilled from zero for every chunk."""
    v, want = data
    ctx.set_tuning(td_fold=2, base2_split=1, base2_ilp=2, rest_window=3, small_max=0,
                   chunk_log2=16)
    try:
        _same(v, _run(ctx, v), want, "chunk_log2=16")
    finally:
        ctx.set_tuning(chunk_log2=24)


def test_variants_on_the_host_path(data, ctx):
    """isprime_u64_host runs the same stages on its two staging slots' own queues."""
    v, want = data
    ctx.set_tuning(td_fold=1, base2_split=1, base2_ilp=2, rest_window=3, small_max=0,
                   chunk_log2=16)
    try:
        _same(v, ctx.isprime_host(v), want, "host path")
    finally:
        ctx.set_tuning(chunk_log2=24)


def test_variants_with_spread_rest_kernel(ctx):
    """Short queues take the six-base kernel that spreads (survivor, base)
    pairs over threads; its 3-bit-window form with the split base-2 queue."""
    rng = random.Random(5)
    pool = [int(x) for x in load_pool("primes_near_2p64.txt")[:500]]
    for n in (7, 64, 1000, 9000):
        vals = [rng.choice(pool) for _ in range(n // 2)] + _spsp_near_2p63(4, seed=n)
        vals += [int(x) for x in plain_large(n - len(vals), seed=n)]
        v = np.array(vals, dtype=np.uint64)
        want = oracle.isprime_u64(v)
        for win in (3, 4):
            ctx.set_tuning(td_fold=2, base2_split=1, base2_ilp=1, rest_window=win, small_max=0)
            _same(v, _run(ctx, v), want, f"spread n={n} win={win}")


@pytest.mark.parametrize("impl,impl_b2,ilp", [(9, 9, 1), (9, 9, 2), (6, 9, 1), (9, 6, 2)])
def test_formulation_9_matches_oracle(impl, impl_b2, ilp, data, ctx):
    """Formulation 9 (the final correction on the multiply pipe) in both stages."""
    v, want = data
    ctx.set_tuning(mont_impl=impl, mont_impl_base2=impl_b2, base2_ilp=ilp, td_fold=2,
                   base2_split=1, rest_window=3, small_max=0, base2_window=1, compact_min=33)
    try:
        _same(v, _run(ctx, v), want, f"impl={impl} impl_b2={impl_b2} ilp={ilp}")
    finally:
        ctx.set_tuning(mont_impl=6, mont_impl_base2=6, base2_ilp=1)


@pytest.mark.parametrize("n", [70001, 1 << 20])
def test_programmatic_dependent_launch_matches_oracle(n, data, ctx):
    """pdl = 1: the Miller-Rabin kernels launched to overlap the kernel before
    them (a short chunk takes the spreading six-base kernel, a long one not)."""
    v, want = data
    reps = -(-n // v.size)
    vv, ww = np.tile(v, reps)[:n], np.tile(want, reps)[:n]
    ctx.set_tuning(pdl=1, small_max=0)
    try:
        _same(vv, _run(ctx, vv), ww, f"pdl n={n}")
    finally:
        ctx.set_tuning(pdl=0)


@pytest.mark.parametrize("n,chunk_log2", [(1 << 20, 24), ((1 << 20) + 12345, 24),
                                           (3 * (1 << 20) + 7, 24), ((1 << 20) + 999, 16)])
def test_dual_stream_matches_oracle(n, chunk_log2, data, ctx):
    """dual_stream = 1: chunks alternate between the caller's stream (first
    queue set) and the context's second stream (second queue set); two
    chunks, or with chunk_log2 = 16 seventeen, a ragged last one.  The call
    runs on a side stream of the caller, whose next kernel must see every
    output; a second call right after reuses both queue sets."""
    v, want = data
    reps = -(-n // v.size)
    vv, ww = np.tile(v, reps)[:n], np.tile(want, reps)[:n]
    ctx.set_tuning(dual_stream=1, small_max=0, chunk_log2=chunk_log2)
    try:
        side = torch.cuda.Stream()
        t = torch.from_numpy(vv.view(np.int64)).to("cuda:0")
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            out1 = ctx.isprime(t)
            s1 = out1.to(torch.int64).sum()      # ordered on the side stream after the call
            out2 = ctx.isprime(t.flip(0))
        torch.cuda.synchronize()
        _same(vv, out1.cpu().numpy(), ww, f"dual n={n} chunk_log2={chunk_log2}")
        _same(vv[::-1], out2.cpu().numpy(), ww[::-1], f"dual second call n={n}")
        assert int(s1) == int(ww.sum())
    finally:
        ctx.set_tuning(dual_stream=0, chunk_log2=24)


def test_dual_stream_double_path_counts_invalid(ctx):
    """The double path in two-stream form: results and the invalid count
    (kernels of both streams add to it) equal the oracle's."""
    rng = np.random.default_rng(77)
    n = (1 << 21) + 3
    d = rng.integers(0, 1 << 53, size=n, endpoint=True).astype(np.float64)
    d[rng.integers(0, n, size=1000)] = 0.5
    d[rng.integers(0, n, size=1000)] = -3.0
    d[rng.integers(0, n, size=10)] = float(1 << 60)
    want, bad = oracle.isprime_f64(d)
    ctx.set_tuning(dual_stream=1, small_max=0, chunk_log2=20)
    try:
        t = torch.from_numpy(d).to("cuda:0")
        inv = torch.zeros(1, dtype=torch.int64, device="cuda:0")
        ctx.f64_status()
        got = ctx.isprime(t, invalid=inv)
        torch.cuda.synchronize()
        _same(d, got.cpu().numpy(), want, "dual f64")
        assert int(inv.item()) == bad
        assert ctx.f64_status() == bad
    finally:
        ctx.set_tuning(dual_stream=0, chunk_log2=24)


TD2_PRIMES = [p for p in range(55, 500, 2) if nt.trial_is_prime(p)][:72]  # 59 .. 457


@pytest.fixture(scope="module")
def td2_data(data):
    """The variant inputs plus values that the second trial stage removes:
    multiples of each of its primes near 2^64, just above 2^32 and at random,
    p q with p one of its primes and q a prime near 2^64 / p, and the same
    with p the first prime after its last group (459 < p: never removed)."""
    v, _ = data
    rng = random.Random(31)
    extra = []
    pool = [int(x) for x in load_pool("primes_near_2p64.txt")[:200]]
    for p in TD2_PRIMES + [461, 463, 467]:
        top = (2**64 - 1) // p
        extra += [p * (top - j) for j in range(6)]
        extra += [p * ((2**32) // p + 1 + j) for j in range(6)]
        extra += [p * rng.randrange(2**32 // p, top) for _ in range(6)]
        q = rng.choice(pool) // p
        while not oracle.isprime1(q):
            q -= 1
        extra.append(p * q)
    w = np.concatenate([v, np.array(extra, dtype=np.uint64)])
    np.random.default_rng(32).shuffle(w)
    return w, oracle.isprime_u64(w)


@pytest.mark.parametrize("td2,split,chunk_log2,window,ilp", [
    (8, 1, 24, 1, 1), (12, 0, 24, 1, 1), (16, 1, 24, 1, 1), (24, 1, 24, 1, 1), (16, 0, 16, 1, 1),
    (24, 1, 16, 1, 1), (16, 1, 24, 2, 1), (0, 1, 24, 2, 1), (16, 0, 16, 2, 1),
    (16, 1, 24, 1, 2), (24, 0, 24, 1, 2), (16, 1, 16, 1, 2), (24, 1, 16, 1, 2), (16, 1, 24, 2, 2),
    (8, 1, 24, 1, 2)])
def test_second_trial_stage_matches_oracle(td2, split, chunk_log2, window, ilp, td2_data, ctx):
    """td2_groups > 0: the base-2 kernel tests its queue against the primes
    59 .. 457 first and stages the survivors per warp; with the s-split on and
    off, one chunk and many (every chunk's stacks drain at its end), and with
    the base-2 window step's quotient estimated in single precision (1) or in
    integers (2); with one staged value per lane or two (base2_ilp 2: batches
    of 64, two interleaved exponentiations per lane)."""
    v, want = td2_data
    ctx.set_tuning(td2_groups=td2, base2_split=split, chunk_log2=chunk_log2, small_max=0,
                   td_fold=2, base2_ilp=ilp, rest_window=3, base2_window=window)
    try:
        _same(v, _run(ctx, v), want,
              f"td2={td2} split={split} chunk_log2={chunk_log2} w={window} ilp={ilp}")
    finally:
        ctx.set_tuning(td2_groups=0, base2_split=1, chunk_log2=24, base2_window=1, base2_ilp=1)


def test_second_trial_stage_on_short_queues(td2_data, ctx):
    """Short queues (the spreading six-base kernel, which relies on the base-2
    kernel's marks) and partial stacks: every length from 1 to 70 and a few
    longer ones, each slice of the inputs on its own."""
    v, want = td2_data
    for ilp in (1, 2):
        ctx.set_tuning(td2_groups=16, small_max=0, base2_ilp=ilp)
        try:
            rng = np.random.default_rng(33)
            for n in list(range(1, 71)) + [127, 1000, 4097, 30001]:
                o = int(rng.integers(0, v.size - n))
                _same(v[o:o + n], _run(ctx, v[o:o + n]), want[o:o + n], f"td2 short n={n} ilp={ilp}")
        finally:
            ctx.set_tuning(td2_groups=0, base2_ilp=1)


@pytest.mark.parametrize("fold", [2, 3])
def test_second_trial_stage_host_and_double_paths(fold, td2_data, ctx):
    v, want = td2_data
    ctx.set_tuning(td2_groups=24, small_max=0, chunk_log2=16, td_fold=fold)
    try:
        _same(v, ctx.isprime_host(v), want, "td2 host path")
        d = (v[:200_000] >> np.uint64(11)).astype(np.float64)  # integers below 2^53
        wd, bad = oracle.isprime_f64(d)
        got = ctx.isprime(torch.from_numpy(d).to("cuda:0"))
        torch.cuda.synchronize()
        assert bad == 0
        _same(d, got.cpu().numpy(), wd, f"td2 double path fold={fold}")
    finally:
        ctx.set_tuning(td2_groups=0, chunk_log2=24, td_fold=2)


@pytest.mark.parametrize("split", [1, 0])
def test_paired_bases_match_oracle(split, td2_data, ctx):
    """rest_ilp = 2 (default): the six-base kernel (its long-queue form, chunks
    above 2^22 values) runs the bases in pairs, two exponentiations per
    thread, and rest_ilp = 1 one base at a time; the
    inputs are the variant set plus plain_large values, 2^22 + 4097 in all,
    so the queue is long and ragged."""
    v0, _ = td2_data
    n = (1 << 22) + 4097
    v = np.concatenate([v0, plain_large(n - v0.size, seed=77)])
    want = oracle.isprime_u64(v)
    for ilp in (2, 1):
        ctx.set_tuning(rest_ilp=ilp, rest_window=3, base2_split=split, small_max=0, chunk_log2=24)
        try:
            _same(v, _run(ctx, v), want, f"rest_ilp={ilp} split={split}")
        finally:
            ctx.set_tuning(rest_ilp=2, base2_split=1)


def test_tuning_rejects_out_of_range_variant_fields(ctx):
    for kw in (dict(td_fold=4), dict(base2_split=2), dict(base2_ilp=3), dict(base2_ilp=0),
               dict(mont_impl=10), dict(mont_impl_base2=10), dict(pdl=2), dict(dual_stream=2),
               dict(td2_groups=4), dict(td2_groups=25), dict(inplace_max_log2=25),
               dict(base2_window=3), dict(serve_long_log2=15), dict(serve_long_log2=29),
               dict(rest_ilp=0), dict(rest_ilp=3),
               dict(rest_window=5), dict(rest_window=2)):
        with pytest.raises(ipg.IsPrimeError):
            ctx.set_tuning(**kw)
