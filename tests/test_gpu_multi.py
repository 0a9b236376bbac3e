"""isprime_u64_host_multi: one host job split over several devices by the
contiguous plan.  This machine gives one GPU, so the device list names
device 0 more than once: the shards then run one after another on it through
the same code (planning, one thread per shard, results in input order).  No
kernels wait on one another.  Results are compared with the CPU oracle."""
import numpy as np
import pytest

import oracle
from workloads import plain_mixed

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402


@pytest.mark.parametrize("devices", [[0], [0, 0], [0, 0, 0]])
@pytest.mark.parametrize("n", [1, 1000, 300_001])
def test_host_multi_matches_oracle(devices, n):
    v = plain_mixed(n, seed=17 + n)
    got = ipg.isprime_host_multi(v, devices)
    want = oracle.isprime_u64(v)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{bad.size} mismatches; first n={int(v[bad[0]])}"
