"""Planning one job across devices (host only, CPU tests).

Every element is independent (Sec. 1), so a job splits across devices with no
exchange of data: contiguous ranges of a plain array, whole arrays of a batch
balanced by size (longest first to the least-loaded shard), and served
requests to the least-loaded device.  The library's planners are checked here
against their stated properties and, on small batches, against the best
possible split found by brute force; two gloo ranks then run a batch split
this way (each rank classifying its share with the oracle) and the union is
compared with the single-process result."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_2108_04791_gb300 as ipg  # noqa: E402


@pytest.mark.parametrize("n,k", [(0, 1), (0, 4), (1, 4), (10, 3), (2**24, 8), (2**40 + 7, 7),
                                 (5, 5), (6, 4)])
def test_contiguous_ranges_cover_and_balance(n, k):
    b = ipg.plan_contiguous(n, k).astype(object)
    assert b[0] == 0 and b[-1] == n and len(b) == k + 1
    sizes = [b[s + 1] - b[s] for s in range(k)]
    assert all(x >= 0 for x in sizes) and max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)  # the remainder goes to the first shards


def _best_makespan(sizes, k):
    best = None
    for assign in itertools.product(range(k), repeat=len(sizes)):
        loads = [0] * k
        for s, a in zip(sizes, assign):
            loads[a] += s
        m = max(loads)
        best = m if best is None else min(best, m)
    return best


def test_batched_plan_against_brute_force_optimum():
    rng = np.random.default_rng(5)
    for trial in range(60):
        k = int(rng.integers(2, 4))
        n = int(rng.integers(1, 8))
        sizes = rng.integers(1, 50, size=n).tolist()
        owner, load = ipg.plan_batched(sizes, k)
        assert owner.size == n and load.size == k
        got = [0] * k
        for s, o in zip(sizes, owner.tolist()):
            got[o] += s
        assert got == load.tolist() and sum(got) == sum(sizes)
        opt = _best_makespan(sizes, k)
        assert 3 * k * max(got) <= (4 * k - 1) * opt  # max <= (4/3 - 1/(3k)) OPT
        assert max(got) <= sum(sizes) / k + max(sizes)


def test_batched_plan_large_ragged_batch_and_ties():
    from workloads import generators as wg
    sizes = wg.log_uniform_sizes(3, 4096, 1 << 20)
    for k in (1, 2, 3, 8):
        owner, load = ipg.plan_batched(sizes, k)
        assert int(load.sum()) == int(sizes.sum())
        assert int(load.max()) <= int(sizes.sum()) / k + int(sizes.max())
        assert np.array_equal(np.bincount(owner, weights=sizes.astype(np.float64), minlength=k),
                              load.astype(np.float64))
    # equal sizes: in index order, each to the least-loaded (lowest) shard
    owner, load = ipg.plan_batched([7] * 6, 3)
    assert owner.tolist() == [0, 1, 2, 0, 1, 2] and load.tolist() == [14, 14, 14]
    owner, load = ipg.plan_batched([], 3)
    assert owner.size == 0 and load.tolist() == [0, 0, 0]


def test_route_least_loaded_and_bad_arguments():
    assert ipg.route_least_loaded([5, 3, 3, 9]) == 1
    assert ipg.route_least_loaded([0]) == 0
    assert ipg.route_least_loaded([2**64 - 1, 2**64 - 2]) == 1
    for call in (lambda: ipg.plan_contiguous(10, 0), lambda: ipg.plan_batched([1, 2], 0),
                 lambda: ipg.route_least_loaded([])):
        with pytest.raises(ipg.IsPrimeError) as e:
            call()
        assert e.value.status == ipg.EINVAL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _batch(seed=11, n_arrays=48):
    from workloads import generators as wg
    sizes = wg.log_uniform_sizes(seed, n_arrays, 4096)
    offs = np.zeros(n_arrays + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    vals = wg.bitlen_uniform(seed, int(offs[-1]), 2, 64)
    return sizes, offs, vals


def _rank_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    sizes, offs, vals = _batch()
    owner, _ = ipg.plan_batched(sizes, world)  # every rank computes the same plan
    mine = {int(a): oracle.isprime_u64(vals[offs[a]:offs[a + 1]], threads=1)
            for a in np.flatnonzero(owner == rank)}
    q.put((rank, mine))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_a_batch_by_plan():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes, offs, vals = _batch()
    done = {}
    for _, mine in parts:
        assert not set(mine) & set(done)  # each array on exactly one rank
        done.update(mine)
    assert sorted(done) == list(range(len(sizes)))
    got = np.concatenate([done[a] for a in range(len(sizes))])
    assert np.array_equal(got, oracle.isprime_u64(vals))


def test_host_multi_rejects_bad_arguments_without_a_device():
    """Argument errors of isprime_u64_host_multi come before any device is used."""
    import ctypes
    L = ipg.lib()
    a = np.arange(10, dtype=np.uint64)
    o = np.zeros(10, dtype=np.uint8)
    d = np.array([0], dtype=np.int32)
    assert L.isprime_u64_host_multi(d.ctypes.data, 0, a.ctypes.data, o.ctypes.data, 10) == ipg.EINVAL
    assert L.isprime_u64_host_multi(None, 1, a.ctypes.data, o.ctypes.data, 10) == ipg.EINVAL
    assert L.isprime_u64_host_multi(d.ctypes.data, 1, None, o.ctypes.data, 10) == ipg.EINVAL
    assert L.isprime_u64_host_multi(d.ctypes.data, 1, a.ctypes.data, o.ctypes.data, 0) == ipg.OK
    bad = np.array([-1], dtype=np.int32)
    assert L.isprime_u64_host_multi(bad.ctypes.data, 1, a.ctypes.data, o.ctypes.data, 10) == ipg.EINVAL
    assert ctypes.c_char_p(L.isprime_last_error()).value
