"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on every output (no sampling): the CPU oracle classifies the
same values on all host cores and the two arrays must be equal byte for byte.

* plain_mixed: all 2^26 uint64 values of the mixed-magnitude workload through
  the default context (and the 2^20 doubles, in tests/test_gpu_parity.py).
* batched: the 4096 ragged arrays (293,037,204 values) in one batched launch.
* served: all 20,000 requests of the served workload through the
  continuous-batching server with four slots.  Each request's values are a
  slice of the 2^27-value pool the benchmark uses, so the oracle classifies
  the pool once and each request's expected bytes are the matching slice;
  the requests go in waves that fit a 2^31-byte output ring, every request of
  a wave is admitted before any is waited for (so they overlap on the GPU),
  and every output byte of every request is compared.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402
from workloads import generators as wg  # noqa: E402
from workloads import torch_gen  # noqa: E402


def _same(vals, got, want, what):
    bad = np.flatnonzero(got != want)
    assert not bad.size, (f"{what}: {bad.size} mismatches; first at {int(bad[0])}: "
                          f"n={int(vals[bad[0]])} gpu={int(got[bad[0]])} "
                          f"oracle={int(want[bad[0]])}")


def test_plain_mixed_full_size():
    v = wg.plain_mixed()
    t = torch.from_numpy(v.view(np.int64)).to("cuda:0")
    got = ipg.isprime(t)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    del t
    _same(v, got, oracle.isprime_u64(v), "plain_mixed 2^26")


def test_batched_full_size():
    dev = torch.device("cuda:0")
    d_all, offs = torch_gen.batched_arrays(n_arrays=4096, max_size=1 << 20, seed=3, device=dev)
    n = d_all.numel()
    assert n == 293_037_204
    out = torch.full((n,), 7, dtype=torch.uint8, device=dev)
    ins = [d_all[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    outs = [out[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    ipg.Context.default(0).isprime_batched(ins, outs=outs)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    vals = d_all.cpu().numpy().view(np.uint64)
    del d_all, out, ins, outs
    _same(vals, got, oracle.isprime_u64(vals), "batched 4096 arrays")


def test_served_all_requests():
    _, sizes, _ = wg.served_requests(n_requests=20_000, max_size=1 << 22, seed=4, values=False)
    pool_n = 1 << 27
    pool = torch_gen.served_values(pool_n, seed=4, device=torch.device("cuda:0")).cpu().pin_memory()
    pool_np = pool.numpy().view(np.uint64)
    want_pool = oracle.isprime_u64(pool_np)
    starts = np.zeros(len(sizes), dtype=np.int64)
    np.cumsum(sizes[:-1], out=starts[1:])
    in_off = starts % (pool_n - (1 << 22))
    ring_n = 1 << 31
    ring = torch.empty(ring_n, dtype=torch.uint8).pin_memory().numpy()
    done = 0
    with ipg.Server(ipg.Context.default(0), mem_budget_bytes=8 << 30, n_slots=4) as srv:
        i = 0
        while i < len(sizes):
            # one wave: consecutive requests whose outputs fit the ring
            j, used = i, 0
            while j < len(sizes) and used + sizes[j] <= ring_n:
                used += int(sizes[j])
                j += 1
            ring[:used] = 7
            offs = np.zeros(j - i + 1, dtype=np.int64)
            np.cumsum(sizes[i:j], out=offs[1:])
            tickets = [srv.submit(pool_np[in_off[k]:in_off[k] + sizes[k]],
                                  out=ring[offs[k - i]:offs[k - i] + sizes[k]]) for k in range(i, j)]
            for t in tickets:
                srv.wait(t)
            for k in range(i, j):
                a, m = int(in_off[k]), int(sizes[k])
                got = ring[offs[k - i]:offs[k - i] + m]
                if not np.array_equal(got, want_pool[a:a + m]):
                    _same(pool_np[a:a + m], got, want_pool[a:a + m], f"request {k}")
            done += j - i
            i = j
    assert done == 20_000
