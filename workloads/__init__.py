"""Seeded synthetic inputs for the primality workloads.

This module holds no primality arithmetic: it only draws random integers.
Both the oracle-side tests and the GPU side (tests, benchmark) take their
inputs from here, so each side sees the same arrays for the same seed.
"""
from .generators import (  # noqa: F401
    splitmix64, uniform_below, uniform_range, bitlen_uniform,
    log_uniform_sizes, plain_small, plain_large, plain_mixed, mixed_doubles,
    batched_arrays, served_requests, load_pool, load_primes_by_bits, WORKLOADS,
)
