"""GPU tests of the continuous-batching server (isprime_server_*).

Each request's result in the mix must equal its result alone (and the
oracle): primality has one answer, so the bar is bit-exactness.  Failure
handling is exercised on the host (budget refusal, a wait that times out,
an unknown ticket, shutdown with work in flight); nothing here faults the
GPU.
"""
import threading

import numpy as np
import pytest

import oracle
from workloads import generators as wg

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402


def _requests(n_req, max_size, seed):
    vals, offs = wg.batched_arrays(n_arrays=n_req, max_size=max_size, seed=seed)
    return [np.ascontiguousarray(vals[offs[i]:offs[i + 1]]) for i in range(n_req)]


@pytest.mark.parametrize("n_slots,small_max,long_log2", [(3, None, 24), (1, None, 24),
                                                        (2, 1 << 12, 24), (3, 0, 24),
                                                        (2, 1 << 10, 16), (3, 0, 16)])
def test_mixed_concurrent_requests_equal_results_alone(n_slots, small_max, long_log2):
    """Short and long requests from four client threads; short ones (at most
    serve_short_max elements) are batched apart and keep the last slot; with
    serve_long_log2 16 a long batch closes at 2^16 values, so many small long
    batches rotate through the slots."""
    reqs = _requests(240, 1 << 15, seed=91) + [np.zeros(0, np.uint64),
                                               np.array([2**64 - 59, 1, 2], np.uint64)]
    ctx = ipg.Context.default(0)
    alone = []
    for r in reqs:  # each request alone, through the plain path
        t = torch.from_numpy(r.view(np.int64)).cuda()
        alone.append(ctx.isprime(t).cpu().numpy() if r.size else np.zeros(0, np.uint8))
    sctx = ipg.Context(0) if small_max is not None else ctx
    if small_max is not None:
        sctx.set_tuning(serve_short_max=small_max, serve_long_log2=long_log2)
    with ipg.Server(sctx, mem_budget_bytes=64 << 20, n_slots=n_slots) as srv:
        results = [None] * len(reqs)

        def client(idx):
            tickets = [(i, srv.submit(reqs[i])) for i in idx]
            for i, t in tickets:
                results[i] = srv.wait(t)

        threads = [threading.Thread(target=client, args=(list(range(k, len(reqs), 4)),))
                   for k in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        st = srv.stats()
    for r, got, a in zip(reqs, results, alone):
        assert np.array_equal(got, a)
        assert np.array_equal(got, oracle.isprime_u64(r))
    assert st["requests"] == len(reqs) and st["elements"] == sum(r.size for r in reqs)
    assert 0 <= st["p50_ms"] <= st["p99_ms"] <= st["max_ms"] and st["tests_per_s"] > 0
    assert 1 <= st["batches"] <= len(reqs)
    if sctx is not ctx:
        sctx.close()


def test_pinned_short_requests_are_served_in_place():
    """Short requests in pinned host memory are read and written by the kernel
    directly (no arena copies); long ones in the same stream of requests are
    copied.  Every result equals the oracle's."""
    reqs = _requests(120, 1 << 14, seed=93)
    pool = torch.empty(sum(r.size for r in reqs), dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    outs = torch.zeros(pool.size + 8 * len(reqs), dtype=torch.uint8).pin_memory().numpy()
    views, ov, a, o = [], [], 0, 0
    for r in reqs:
        pool[a:a + r.size] = r
        views.append(pool[a:a + r.size])
        ov.append(outs[o + 1:o + 1 + r.size])  # odd output offsets
        a += r.size
        o += r.size + 8
    ctx = ipg.Context(0)
    ctx.set_tuning(serve_short_max=1 << 12)
    with ipg.Server(ctx, mem_budget_bytes=32 << 20, n_slots=2) as srv:
        tickets = [srv.submit(v, out=w) for v, w in zip(views, ov)]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    ctx.close()
    for r, g_ in zip(reqs, got):
        assert np.array_equal(g_, oracle.isprime_u64(r))
    assert st["short_requests"] == sum(1 for r in reqs if r.size <= 1 << 12) > 0
    assert st["p50_short_ms"] <= st["p99_short_ms"]


def test_budget_refusal_unknown_ticket_and_timeout():
    ctx = ipg.Context.default(0)
    big = _requests(1, 1 << 12, seed=92)[0]
    budget = 1 << 20  # 1 MiB: room for one request of ~100k elements at a time
    with ipg.Server(ctx, mem_budget_bytes=budget, n_slots=1) as srv:
        with pytest.raises(ipg.IsPrimeError) as e:
            srv.submit(np.arange(200_000, dtype=np.uint64))
        assert e.value.status == ipg.EBUSY
        with pytest.raises(ipg.IsPrimeError) as e:
            srv.wait(123456789, 0)
        assert e.value.status == ipg.EINVAL
        # two requests that cannot share the budget: the second starts only
        # after the first finished, so it is still pending right after submit
        pool = wg.load_pool("primes_near_2p64.txt")
        heavy = np.resize(pool, 100_000)
        t1 = srv.submit(heavy)
        t2 = srv.submit(heavy.copy())
        with pytest.raises(ipg.IsPrimeError) as e:
            srv.wait(t2, 0)
        assert e.value.status == ipg.ETIMEDOUT
        assert srv.wait(t1).all() and srv.wait(t2).all()  # every value is a prime
        out = srv.wait(srv.submit(big))
        assert np.array_equal(out, oracle.isprime_u64(big))


def test_shutdown_finishes_admitted_requests():
    ctx = ipg.Context.default(0)
    reqs = _requests(64, 1 << 14, seed=93)
    outs = [np.full(r.size, 7, np.uint8) for r in reqs]
    srv = ipg.Server(ctx, mem_budget_bytes=32 << 20, n_slots=2)
    for r, o in zip(reqs, outs):
        srv.submit(r, out=o)
    srv.close()  # must drain before returning
    for r, o in zip(reqs, outs):
        assert np.array_equal(o, oracle.isprime_u64(r))
