"""The seeded generators: the torch version reproduces the numpy version
bit for bit, and the distributions have the stated shapes.  CPU only."""
import numpy as np
import pytest

import workloads.generators as g

torch = pytest.importorskip("torch")
import workloads.torch_gen as tg  # noqa: E402


def _u(t):
    return t.numpy().view(np.uint64)


def test_splitmix_and_mappings_match_numpy():
    for seed in (0, 1, 2, 12345):
        assert np.array_equal(_u(tg.splitmix64(seed, 5000, 77, "cpu")), g.splitmix64(seed, 5000, 77))
    assert np.array_equal(_u(tg.uniform_range(1, 5000, 1 << 49, 1 << 64, 3, "cpu")),
                          g.uniform_range(1, 5000, 1 << 49, 1 << 64, 3))
    assert np.array_equal(_u(tg.uniform_range(0, 5000, 0, 10**6, 0, "cpu")),
                          g.uniform_range(0, 5000, 0, 10**6))
    assert np.array_equal(_u(tg.bitlen_uniform(2, 20000, 2, 64, 5, "cpu")),
                          g.bitlen_uniform(2, 20000, 2, 64, 5))


def test_batched_values_match_numpy():
    v, offs = tg.batched_arrays(n_arrays=50, max_size=1 << 12, seed=9, device="cpu")
    w, offs2 = g.batched_arrays(n_arrays=50, max_size=1 << 12, seed=9)
    assert np.array_equal(offs, offs2)
    assert np.array_equal(_u(v), w)


def test_distribution_shapes():
    v = g.plain_large(1 << 16)
    assert v.min() >= 1 << 49 and (v[0::2] & np.uint64(1)).all()
    m = g.plain_mixed(1 << 16)
    bl = np.array([int(x).bit_length() for x in m])
    assert bl.min() == 2 and bl.max() == 64
    counts = np.bincount(bl)[2:]
    assert counts.min() > 0.7 * counts.mean()
    s = g.log_uniform_sizes(3, 4096, 1 << 20)
    assert s.min() >= 1 and s.max() <= 1 << 20
    vals, offs = g.batched_arrays(n_arrays=40, max_size=1 << 12, seed=5)
    pools = set(g.load_pool("primes_near_2p64.txt").tolist())
    frac = np.isin(vals, np.array(sorted(pools), dtype=np.uint64)).mean()
    assert 0.2 < frac < 0.3
    arr, sizes, _ = g.served_requests(n_requests=2000, values=False)
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 5000) < 0.1 / 5000


def test_stored_primes_by_bits_have_their_bit_size_and_are_prime():
    """Table 4's scalar inputs: 100 primes per bit size, each in [2^(b-1), 2^b);
    primality re-checked by trial division (<= 32 bits) or a Pratt certificate."""
    import numtheory as nt
    pools = g.load_primes_by_bits()
    assert sorted(pools) == [4, 8, 16, 24, 32, 36, 40, 44, 48, 50, 52, 56, 60, 64]
    for b, vals in pools.items():
        assert vals.size == 100
        for v in vals.tolist():
            assert v.bit_length() == b
        for v in sorted(set(vals.tolist()))[:5]:
            if b <= 32:
                assert nt.trial_is_prime(v)
            else:
                assert nt.pratt_prime(v) is True
