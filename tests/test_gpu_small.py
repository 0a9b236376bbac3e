"""GPU parity of the latency path (one warp per element, one launch).

Scalars through isprime_u64_scalar, host arrays of up to
ISPRIME_HOST_INLINE_MAX values through isprime_u64_host (values in the
kernel parameters, results in mapped host memory), and device arrays of up
to `small_max` elements through isprime_u64_ctx / isprime_f64_ctx.  Every
answer is compared with the CPU oracle, bit for bit, and with the queue
path of the same context (small_max = 0).
"""
import numpy as np
import pytest

import oracle
from workloads import plain_mixed, plain_large, load_primes_by_bits

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402

INLINE_MAX = 256

SPECIAL = [0, 1, 2, 3, 4, 5, 9, 15, 25, 49, 241, 251, 253, 255, 257, 263, 66047, 66049, 66053,
           257 * 263, 65521, 65537, 561, 1105, 1729, 2047, 3277, 4033, 4681, 8321, 25326001,
           3215031751, 2152302898747, 3474749660383, 341550071728321, 3825123056546413051,
           318665857834031151167461, 2**31 - 1, 2**32 - 5, 2**32 - 1, 2**32, 2**32 + 1,
           2**32 + 15, 4759123141, 1122004669633, 2**48 - 59, 2**52 - 47, 2**53 - 111,
           2**61 - 1, 2**62 - 57, 2**63 - 25, 2**63, 2**63 + 1, 2**64 - 59, 2**64 - 57,
           2**64 - 3, 2**64 - 1]
SPECIAL = [v for v in SPECIAL if v < 1 << 64]


def _dev():
    return torch.device("cuda:0")


def _to_dev(vals):
    return torch.from_numpy(np.ascontiguousarray(vals, dtype=np.uint64).view(np.int64)).to(_dev())


@pytest.fixture(scope="module", params=["default", "nosieve", "sieve2p20"])
def ctx(request):
    if request.param == "default":
        yield ipg.Context.default(0)
    else:
        with ipg.Context(0, sieve_limit=0 if request.param == "nosieve" else 1 << 20) as c:
            yield c


def _stress_values():
    """Base-2 strong pseudoprimes, Carmichael numbers (6k+1)(12k+1)(18k+1)
    and semiprimes of primes near 2^32: composites the warp path must reject."""
    import numtheory as nt
    comp = ~nt.simple_sieve(300_000)
    spsp = [n for n in range(9, 300_000, 2) if comp[n] and nt.strong_base2(n)]
    cars = []
    for k in range(1, 4000):
        a, b, c = 6 * k + 1, 12 * k + 1, 18 * k + 1
        if nt.trial_is_prime(a) and nt.trial_is_prime(b) and nt.trial_is_prime(c):
            cars.append(a * b * c)
    p = [int(x) for x in load_primes_by_bits()[32][:20]]
    semi = [p[i] * p[i + 1] for i in range(19)]
    return np.array(spsp + cars + semi, dtype=np.uint64)


def test_scalar_special_values(ctx):
    want = oracle.isprime_u64(np.array(SPECIAL, dtype=np.uint64))
    got = [ctx.isprime_scalar(v) for v in SPECIAL]
    assert got == [bool(w) for w in want.tolist()], [v for v, g_, w in zip(SPECIAL, got, want) if g_ != w]


def test_scalar_table4_primes_every_bit_size(ctx):
    for b, vals in load_primes_by_bits().items():
        got = [ctx.isprime_scalar(int(v)) for v in vals[:25]]
        assert all(got), (b, [int(v) for v, g_ in zip(vals, got) if not g_])
        # the odd neighbours v + 2 and v - 2 are mostly composite
        nb = np.array([int(v) + 2 for v in vals[:25] if int(v) + 2 < 1 << b], dtype=np.uint64)
        want = oracle.isprime_u64(nb)
        assert [ctx.isprime_scalar(int(v)) for v in nb] == [bool(w) for w in want.tolist()], b


def test_scalar_rejects_pseudoprimes(ctx):
    v = _stress_values()
    for x in v[::7].tolist():
        assert ctx.isprime_scalar(x) is False, x


def test_host_inline_sizes(ctx):
    v = np.concatenate([np.array(SPECIAL, dtype=np.uint64), plain_mixed(400, seed=71)])
    want_all = oracle.isprime_u64(v)
    for n in (1, 2, 3, 4, 5, 31, 32, 33, 100, INLINE_MAX - 1, INLINE_MAX, INLINE_MAX + 1, 400):
        got = ctx.isprime_host(v[:n])
        assert got.tolist() == want_all[:n].tolist(), n


def test_device_small_path_equals_queue_path_and_oracle():
    v = np.concatenate([np.array(SPECIAL, dtype=np.uint64), _stress_values(),
                        plain_large(3000, seed=72), plain_mixed(3000, seed=73)])
    want = oracle.isprime_u64(v)
    for S, cut in ((0, 32), (1 << 20, 32), (1 << 32, 32), (1 << 32, 17), (1 << 32, 0)):
        with ipg.Context(0, sieve_limit=S) as c:
            for small_max in (0, 1 << 20):
                c.set_tuning(small_max=small_max, sieve_cutover_log2=cut)
                for n in (1, 2, 5, 64, 1000, v.size):
                    t = _to_dev(v[:n])
                    out = torch.full((n + 1,), 7, dtype=torch.uint8, device=_dev())[1:]
                    c.isprime(t, out=out)
                    torch.cuda.synchronize()
                    assert out.cpu().numpy().tolist() == want[:n].tolist(), (S, small_max, n)


def test_device_small_path_ragged_offsets():
    base = plain_mixed(2048, seed=74)
    big = _to_dev(base)
    want = oracle.isprime_u64(base)
    with ipg.Context(0) as c:
        c.set_tuning(small_max=1 << 20)
        for off in (0, 1, 3):
            for n in list(range(1, 40)) + [127, 129, 1025, 2045]:
                out = torch.zeros(n + 3, dtype=torch.uint8, device=_dev())[1:n + 1]
                c.isprime(big[off:off + n], out=out)
                torch.cuda.synchronize()
                assert out.cpu().numpy().tolist() == want[off:off + n].tolist(), (off, n)


def test_device_small_path_f64_invalid_count():
    x = np.array([0.0, -0.0, 1.0, 2.0, 7.0, 9.0, 2.0**53, 2.0**53 - 111, float("nan"),
                  float("inf"), -float("inf"), -7.0, 2.5, 2.0**53 + 2, 1e300, 97.0, 3.0,
                  4503599627370449.0], dtype=np.float64)
    c = ipg.Context.default(0)
    for k in (1, 2, 9, len(x)):
        t = torch.from_numpy(x[:k].copy()).to(_dev())
        inv = torch.zeros(1, dtype=torch.int64, device=_dev())
        out = c.isprime(t, invalid=inv)
        torch.cuda.synchronize()
        want, bad = oracle.isprime_f64(x[:k])
        assert out.cpu().numpy().tolist() == want.tolist()
        assert int(inv.item()) == bad


def test_small_path_is_one_launch_and_records_timing():
    c = ipg.Context.default(0)
    assert c.tuning.small_max >= 500
    c.timing_reset()
    c.timing(True)
    c.isprime(_to_dev(plain_large(500, seed=75)))
    c.isprime_scalar(2**64 - 59)
    c.isprime_host(np.arange(100, dtype=np.uint64))
    torch.cuda.synchronize()
    rec = c.timing_read()
    c.timing(False)
    assert rec["small"][1] == 3
    assert rec["classify_u64"][1] == 0 and rec["mr64_base2"][1] == 0


def test_small_max_bounds():
    c = ipg.Context.default(0)
    old = c.tuning.small_max
    with pytest.raises(ipg.IsPrimeError):
        c.set_tuning(small_max=(1 << 20) + 1)
    assert c.tuning.small_max == old


def test_scalar_threads_share_a_context():
    import threading
    vals = [int(v) for v in load_primes_by_bits()[64][:40]] + [int(x) for x in _stress_values()[:40]]
    want = [bool(w) for w in oracle.isprime_u64(np.array(vals, dtype=np.uint64)).tolist()]
    c = ipg.Context.default(0)
    res = [None] * 4

    def work(k):
        res[k] = [c.isprime_scalar(v) for v in vals]

    th = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert all(r == want for r in res)
