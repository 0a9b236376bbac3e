"""CPU oracle for elementwise primality (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product library never loads it, and it shares no
code with the CUDA path.  The arithmetic lives in ``isprime_oracle.c`` (plain
C, compiled with gcc); this module only builds it and marshals numpy arrays
through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isprime_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u64, sz, p = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_void_p
            L.oracle_mulmod.argtypes = [u64, u64, u64]
            L.oracle_mulmod.restype = u64
            L.oracle_mulmod_classic.argtypes = [u64, u64, u64]
            L.oracle_mulmod_classic.restype = u64
            L.oracle_modadd.argtypes = [u64, u64, u64]
            L.oracle_modadd.restype = u64
            L.oracle_powmod.argtypes = [u64, u64, u64]
            L.oracle_powmod.restype = u64
            L.oracle_sprp.argtypes = [u64, u64]
            L.oracle_sprp.restype = ctypes.c_int
            L.oracle_isprime1.argtypes = [u64]
            L.oracle_isprime1.restype = ctypes.c_int
            L.oracle_isprime_u64.argtypes = [p, p, sz]
            L.oracle_isprime_u64.restype = None
            L.oracle_isprime_u64_mt.argtypes = [p, p, sz, ctypes.c_int]
            L.oracle_isprime_u64_mt.restype = None
            L.oracle_isprime_f64.argtypes = [p, p, sz]
            L.oracle_isprime_f64.restype = u64
            L.oracle_count_primes.argtypes = [u64, u64, ctypes.c_int]
            L.oracle_count_primes.restype = u64
            L.oracle_primes_upto.argtypes = [u64, p, sz]
            L.oracle_primes_upto.restype = sz
            L.oracle_isprime_division_count.argtypes = [u64]
            L.oracle_isprime_division_count.restype = u64
            L.oracle_wheel_diffs_mod.argtypes = [u64, p, ctypes.c_int]
            L.oracle_wheel_diffs_mod.restype = ctypes.c_int
            L.oracle_wheel_diffs.argtypes = [p]
            L.oracle_wheel_diffs.restype = ctypes.c_int
            L.oracle_isprime_wheel.argtypes = [u64]
            L.oracle_isprime_wheel.restype = ctypes.c_int
            L.oracle_work_counts.argtypes = [p, sz, ctypes.c_uint32, u64, p]
            L.oracle_work_counts.restype = None
            _lib = L
    return _lib


def _threads(threads):
    if threads is None or threads <= 0:
        return os.cpu_count() or 1
    return threads


def isprime_u64(values, threads: int | None = None) -> np.ndarray:
    """out[i] = 1 iff values[i] is prime (uint8, same shape)."""
    a = np.ascontiguousarray(values, dtype=np.uint64)
    out = np.empty(a.shape, dtype=np.uint8)
    L = lib()
    if a.size:
        L.oracle_isprime_u64_mt(a.ctypes.data, out.ctypes.data, a.size,
                                _threads(threads))
    return out


def isprime_f64(values):
    """Returns (out uint8, invalid_count) for a double array."""
    a = np.ascontiguousarray(values, dtype=np.float64)
    out = np.empty(a.shape, dtype=np.uint8)
    bad = lib().oracle_isprime_f64(a.ctypes.data, out.ctypes.data, a.size) if a.size else 0
    return out, int(bad)


def isprime1(n: int) -> bool:
    return bool(lib().oracle_isprime1(n))


def count_primes(lo: int, hi: int, threads: int | None = None) -> int:
    """Number of primes in [lo, hi)."""
    return int(lib().oracle_count_primes(lo, hi, _threads(threads)))


def primes_upto(N: int) -> np.ndarray:
    L = lib()
    k = L.oracle_primes_upto(N, None, 0)
    out = np.empty(k, dtype=np.uint64)
    if k:
        L.oracle_primes_upto(N, out.ctypes.data, k)
    return out


def division_count(N: int) -> int:
    return int(lib().oracle_isprime_division_count(N))


def wheel_diffs() -> list[int]:
    buf = (ctypes.c_uint32 * 48)()
    k = lib().oracle_wheel_diffs(buf)
    assert k == 48, k
    return list(buf)


def wheel_diffs_mod(P: int) -> list[int]:
    """Difference cycle of the wheel with modulus P (Sec. 3)."""
    k = lib().oracle_wheel_diffs_mod(P, None, 0)
    buf = (ctypes.c_uint32 * max(k, 1))()
    lib().oracle_wheel_diffs_mod(P, buf, k)
    return list(buf)[:k]


def isprime_wheel(n: int) -> bool:
    return bool(lib().oracle_isprime_wheel(n))


def mulmod(a, b, m):
    return int(lib().oracle_mulmod(a, b, m))


def mulmod_classic(a, b, m):
    return int(lib().oracle_mulmod_classic(a, b, m))


def modadd(a, b, m):
    return int(lib().oracle_modadd(a, b, m))


def powmod(a, e, m):
    return int(lib().oracle_powmod(a, e, m))


def sprp(n, a) -> bool:
    return bool(lib().oracle_sprp(n, a))


WORK_KEYS = ("mr64_elements", "base2_squarings", "base2_doublings", "base2_passes",
             "rest_squarings", "rest_multiplies", "base_tests", "trial_tests",
             "mr32_elements", "primes")


def work_counts(values, td_bound: int = 53, sieve_limit: int = 1 << 32) -> dict:
    """Counts of the method's modular operations over the array."""
    a = np.ascontiguousarray(values, dtype=np.uint64)
    c = np.zeros(len(WORK_KEYS), dtype=np.uint64)
    lib().oracle_work_counts(a.ctypes.data, a.size, td_bound, sieve_limit,
                             c.ctypes.data)
    return {k: int(v) for k, v in zip(WORK_KEYS, c)}
