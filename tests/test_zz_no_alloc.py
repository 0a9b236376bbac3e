"""GPU test of isprime_u64_noalloc, the entry point that allocates nothing.

It is for callers that cannot call cudaMalloc when they need the test (for
example code running under an allocator that owns all device memory), so it
keeps its queues in a fixed device array inside the library.  This test
calls it through the C ABI and compares its output with the existing
isprime_u64 entry point (bit-exact: primality has one right answer), on
two calls in a row, so that the second call also shows that the shared
array's leftover contents from the first call do not leak into results.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from workloads import plain_large, plain_mixed

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300 as ipg  # noqa: E402

MAX_ELEMS = 1 << 20


def _lib():
    L = ipg.lib()
    f = L.isprime_u64_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def _run(fn_name, t):
    L = _lib()
    out = torch.full((t.numel(),), 7, dtype=torch.uint8, device=t.device)
    stream = torch.cuda.current_stream(t.device)
    st = getattr(L, fn_name)(t.data_ptr(), out.data_ptr(), t.numel(),
                             ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, (st, L.isprime_last_error())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.uint64).view(np.int64)).to("cuda:0")


def test_noalloc_matches_isprime_u64_two_calls_in_a_row():
    special = np.array([0, 1, 2, 3, 4, 97, 561, 2047, 65537, 4759123141, 2**32 - 5,
                        2**32 + 15, 2**61 - 1, 2**64 - 59, 2**64 - 1], dtype=np.uint64)
    # first call: a full-size array of mixed magnitudes (exercises both queues)
    v1 = np.concatenate([special, plain_mixed(MAX_ELEMS - special.size, seed=71)])
    # second call: a smaller array of large values
    v2 = plain_large(300_001, seed=72)
    for v in (v1, v2):
        t = _dev(v)
        got = _run("isprime_u64_noalloc", t)
        want = _run("isprime_u64", t)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, f"{bad.size} mismatches, first n={int(v[bad[0]])}"
        assert set(np.unique(got).tolist()) <= {0, 1}
        # and against the CPU oracle directly: the special values plus a few
        # thousand of the array (the two entry points share classify and the
        # Montgomery arithmetic, so this check does not lean on isprime_u64)
        k = np.r_[np.arange(min(v.size, 4096)), np.arange(max(0, v.size - 4096), v.size)]
        ref = oracle.isprime_u64(v[k])
        bad = np.flatnonzero(got[k] != ref)
        assert bad.size == 0, f"oracle: {bad.size} mismatches, first n={int(v[k][bad[0]])}"


def test_noalloc_limits():
    L = _lib()
    t = torch.zeros(8, dtype=torch.int64, device="cuda:0")
    o = torch.zeros(8, dtype=torch.uint8, device="cuda:0")
    assert L.isprime_u64_noalloc(t.data_ptr(), o.data_ptr(), 0, None) == 0
    st = L.isprime_u64_noalloc(t.data_ptr(), o.data_ptr(), MAX_ELEMS + 1, None)
    assert st == ipg.EINVAL
    assert b"ISPRIME_NOALLOC_MAX_ELEMS" in L.isprime_last_error()
