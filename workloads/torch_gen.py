"""The generators of `generators.py`, computed with torch on any device.

Same counter-based splitmix64 streams and the same integer mappings, so the
values are bit-identical to the numpy version (tests/test_workloads.py
checks this on the CPU); the GPU runs them fast enough for the large
batched and served workloads.  uint64 bit patterns are held in int64
tensors: additions and multiplications wrap identically, and logical right
shifts are emulated with a mask.  Array sizes (a few thousand values that
go through exp/log) are still drawn by the numpy version.
"""
from __future__ import annotations

import numpy as np
import torch

from . import generators as g

_MASK32 = 0xFFFFFFFF


def _i64(u: int) -> int:
    """uint64 constant -> int64 with the same bits."""
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= 1 << 63 else u


_G = _i64(g.GOLDEN)
_M1 = _i64(0xBF58476D1CE4E5B9)
_M2 = _i64(0x94D049BB133111EB)


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed: int, n: int, offset: int = 0, device="cuda") -> torch.Tensor:
    base = _i64(seed * g.GOLDEN)
    i = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    z = base + i * _G
    z = (z ^ _lsr(z, 30)) * _M1
    z = (z ^ _lsr(z, 27)) * _M2
    return z ^ _lsr(z, 31)


def mulhi64(a: torch.Tensor, b) -> torch.Tensor:
    if not torch.is_tensor(b):
        b = torch.full_like(a, _i64(int(b)))
    a0, a1 = a & _MASK32, _lsr(a, 32)
    b0, b1 = b & _MASK32, _lsr(b, 32)
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = _lsr(p00, 32) + (p01 & _MASK32) + (p10 & _MASK32)
    return p11 + _lsr(p01, 32) + _lsr(p10, 32) + _lsr(mid, 32)


def uniform_range(seed: int, n: int, lo: int, hi: int, offset: int = 0, device="cuda"):
    r = splitmix64(seed, n, offset, device)
    span = hi - lo
    if span >= 1 << 64:
        return r
    return _i64(lo) + mulhi64(r, span)


def bitlen_uniform(seed: int, n: int, lo_bits: int = 2, hi_bits: int = 64, offset: int = 0,
                   device="cuda") -> torch.Tensor:
    r1 = splitmix64(seed, n, offset, device)
    r2 = splitmix64(seed ^ 0x5DEECE66D, n, offset, device)
    b = mulhi64(r1, hi_bits - lo_bits + 1) + lo_bits
    half = torch.ones_like(b) << (b - 1)
    return half + mulhi64(r2, half)


def _replace_with_pools(v: torch.Tensor, seed: int) -> torch.Tensor:
    n = v.numel()
    dev = v.device
    big = torch.from_numpy(g.load_pool("primes_near_2p64.txt").view(np.int64)).to(dev)
    small = torch.from_numpy(g.load_pool("primes_near_2p32.txt").view(np.int64)).to(dev)
    r = splitmix64(seed ^ 0xBA7C4, n, 0, dev)
    u = _lsr(r, 11).to(torch.float64) * (1.0 / (1 << 53))
    pick = splitmix64(seed ^ 0x9001, n, 0, dev)
    pick2 = splitmix64(seed ^ 0x9002, n, 0, dev)
    is_p = u < 0.25
    is_sp = (u >= 0.25) & (u < 0.35)
    v = v.clone()
    v[is_p] = big[mulhi64(pick[is_p], big.numel())]
    p = small[mulhi64(pick[is_sp], small.numel())]
    q = small[mulhi64(pick2[is_sp], small.numel())]
    v[is_sp] = p * q
    return v


def batched_arrays(n_arrays: int = 4096, max_size: int = 1 << 20, seed: int = 3, device="cuda"):
    """(values as an int64 tensor holding uint64 bits, offsets numpy array)."""
    sizes = g.log_uniform_sizes(seed, n_arrays, max_size)
    offsets = np.zeros(n_arrays + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    v = bitlen_uniform(seed, int(offsets[-1]), 2, 64, 0, device)
    return _replace_with_pools(v, seed), offsets


def served_values(total: int, seed: int = 4, device="cuda") -> torch.Tensor:
    """The values of served_requests(), concatenated in request order."""
    return _replace_with_pools(bitlen_uniform(seed, total, 2, 64, 0, device), seed)
