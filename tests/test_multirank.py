"""Multi-rank plumbing on the CPU (gloo, world size 2, 127.0.0.1).

The path shards without a collective: each rank takes its own contiguous
block of the counter-based input stream and classifies it alone; the only
cross-rank steps are the benchmark's barrier and max-over-ranks timing."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    m = bench._max_over_ranks(float(10 + rank), world)
    bench._barrier(world)
    v, _ = bench._workload("plain_large", rank)
    shard = v[:4096]
    out = oracle.isprime_u64(shard, threads=1)
    q.put((rank, m, shard, out))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, s0, o0), (r1, m1, s1, o1) = res
    assert m0 == m1 == 11.0
    # shards are consecutive blocks of one counter-based stream
    from workloads import generators as g
    both = g.uniform_range(1, 2 << 24, 1 << 49, 1 << 64)
    both[0::2] |= np.uint64(1)
    assert np.array_equal(s0, both[:4096])
    assert np.array_equal(s1, both[1 << 24:(1 << 24) + 4096])


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0
