"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on sampled outputs the oracle computes one by one.

* batched: the 4096 ragged arrays (2.9e8 values) in one batched launch;
  2^20 positions sampled uniformly over the whole batch, plus every array's
  first and last element.
* served: the first 400 requests of the served workload (their values are the
  bench's pool slices, in pinned host memory) through the continuous-batching
  server with four slots; 2^20 sampled positions plus every request's ends.
* plain_mixed: covered by tests/test_gpu_parity.py (every 61st value of 2^26).
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


def _check_sample(values_u64, got, pos):
    want = oracle.isprime_u64(values_u64[pos])
    bad = np.flatnonzero(got[pos] != want)
    assert not bad.size, (f"{bad.size} mismatches; first n={int(values_u64[pos[bad[0]]])} "
                          f"gpu={int(got[pos[bad[0]]])} oracle={int(want[bad[0]])}")


def test_batched_full_size_sampled():
    dev = torch.device("cuda:0")
    d_all, offs = torch_gen.batched_arrays(n_arrays=4096, max_size=1 << 20, seed=3, device=dev)
    n = d_all.numel()
    out = torch.full((n,), 7, dtype=torch.uint8, device=dev)
    ins = [d_all[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    outs = [out[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    ipg.Context.default(0).isprime_batched(ins, outs=outs)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    vals = d_all.cpu().numpy().view(np.uint64)
    assert got.max() <= 1  # every byte written
    rng = np.random.default_rng(5)
    pos = np.concatenate([rng.integers(0, n, 1 << 20), offs[:-1][np.diff(offs) > 0],
                          offs[1:][np.diff(offs) > 0] - 1])
    _check_sample(vals, got, pos)


def test_served_prefix_sampled():
    _, sizes, _ = wg.served_requests(n_requests=20_000, max_size=1 << 22, seed=4, values=False)
    sizes = sizes[:400]
    pool_n = 1 << 27
    pool = torch_gen.served_values(pool_n, seed=4, device=torch.device("cuda:0")).cpu().pin_memory()
    pool_np = pool.numpy().view(np.uint64)
    starts = np.zeros(len(sizes), dtype=np.int64)
    np.cumsum(sizes[:-1], out=starts[1:])
    in_off = starts % (pool_n - (1 << 22))
    total = int(sizes.sum())
    out = torch.full((total,), 7, dtype=torch.uint8).pin_memory().numpy()
    with ipg.Server(ipg.Context.default(0), mem_budget_bytes=8 << 30, n_slots=4) as srv:
        tickets = [srv.submit(pool_np[in_off[i]:in_off[i] + sizes[i]],
                              out=out[starts[i]:starts[i] + sizes[i]]) for i in range(len(sizes))]
        for t in tickets:
            srv.wait(t)
    assert out.max() <= 1
    vals = np.concatenate([pool_np[in_off[i]:in_off[i] + sizes[i]] for i in range(len(sizes))])
    rng = np.random.default_rng(6)
    pos = np.concatenate([rng.integers(0, total, 1 << 20), starts, starts + sizes - 1])
    _check_sample(vals, out, pos)
