"""GB300 elementwise primality (isprime) -- thin Python binding.

Every step of the computation runs in the CUDA library
(_lib/libisprime_gb300.so, C ABI in include/isprime.h); this module only
marshals arguments: torch supplies device memory and the current stream.
There is no CPU fallback: if the library is not built, every call raises.

    import torch, paper_2108_04791_gb300 as ip
    x = torch.tensor([1, 2, 3, 4, 5], dtype=torch.int64, device="cuda")
    ip.isprime(x)            # tensor([0, 1, 1, 0, 1], dtype=torch.uint8)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["build", "lib", "isprime", "isprime_host", "isprime_scalar", "Context", "Server", "Tuning",
           "IsPrimeError", "int_rates", "KERNEL_NAMES", "plan_contiguous", "plan_batched",
           "route_least_loaded"]

_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, EDOMAIN, ETIMEDOUT, EBUSY = 0, -1, -2, -3, -4, -5, -6
SIEVE_DEFAULT = (1 << 64) - 1
KERNEL_NAMES = ["sieve_base", "sieve_segment", "classify_u64", "classify_f64",
                "mr64_base2", "mr64_rest", "mr32", "sieve_count", "batched", "range", "small"]


class IsPrimeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"isprime error {status}: {msg}")
        self.status = status


class Tuning(ctypes.Structure):
    _fields_ = [("classify_block", ctypes.c_uint32), ("mr_block", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("td_primes", ctypes.c_uint32),
                ("chunk_log2", ctypes.c_uint32), ("mont_impl", ctypes.c_uint32),
                ("mont_impl_base2", ctypes.c_uint32), ("batch_block", ctypes.c_uint32),
                ("batch_tile_log2", ctypes.c_uint32), ("batch_blocks_per_sm", ctypes.c_uint32),
                ("base2_window", ctypes.c_uint32), ("rest_test", ctypes.c_uint32),
                ("small_max", ctypes.c_uint32), ("compact_min", ctypes.c_uint32),
                ("sieve_cutover_log2", ctypes.c_uint32), ("serve_short_max", ctypes.c_uint32),
                ("td_fold", ctypes.c_uint32), ("base2_split", ctypes.c_uint32),
                ("base2_ilp", ctypes.c_uint32), ("rest_window", ctypes.c_uint32),
                ("window_ratio16", ctypes.c_uint32), ("base2_blocks_per_sm", ctypes.c_uint32),
                ("pdl", ctypes.c_uint32), ("td2_groups", ctypes.c_uint32),
                ("dual_stream", ctypes.c_uint32), ("host_chunk_log2", ctypes.c_uint32),
                ("inplace_max_log2", ctypes.c_uint32), ("serve_long_log2", ctypes.c_uint32),
                ("rest_ilp", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ArrayDesc(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("elements", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("span_s", ctypes.c_double),
                ("tests_per_s", ctypes.c_double), ("short_requests", ctypes.c_uint64),
                ("p50_short_ms", ctypes.c_double), ("p99_short_ms", ctypes.c_double),
                ("p50_long_ms", ctypes.c_double), ("p99_long_ms", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_uint64), ("elements", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("sieve_limit", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_uint64), ("window_calls", ctypes.c_uint64)]


class _OpCounts(ctypes.Structure):
    _fields_ = [("elements", ctypes.c_uint64), ("base2_squarings", ctypes.c_uint64 * 2),
                ("base2_products", ctypes.c_uint64 * 2), ("base2_steps", ctypes.c_uint64 * 2),
                ("rest_squarings", ctypes.c_uint64 * 2), ("rest_products", ctypes.c_uint64 * 2)]


class _KTime(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double), ("launches", ctypes.c_uint64)]


class _IntRates(ctypes.Structure):
    _fields_ = [("mad_lo_u32", ctypes.c_double), ("mad_hi_u32", ctypes.c_double),
                ("mad_wide_u32", ctypes.c_double), ("mont_variant", ctypes.c_double * 10),
                ("sm_clock_mhz", ctypes.c_double)]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the CUDA library for sm_103a (in-tree)."""
    return _build.build(force=force, verbose=verbose)


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            # ISPRIME_GB300_LIB selects another build of the same library (the
            # debug build with bounds checks, see _build.build(debug=True))
            path = os.environ.get("ISPRIME_GB300_LIB") or _build.LIB_PATH
            if not os.path.exists(path):
                raise IsPrimeError(ECUDA, f"CUDA library not built ({path}); run "
                                   "paper_2108_04791_gb300.build() on a machine with nvcc")
            L = ctypes.CDLL(path)
            vp, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
            sigs = {
                "isprime_ctx_create": ([i32, u64, ctypes.POINTER(vp)], i32),
                "isprime_ctx_destroy": ([vp], i32),
                "isprime_default_ctx": ([i32, ctypes.POINTER(vp)], i32),
                "isprime_ctx_get_tuning": ([vp, ctypes.POINTER(Tuning)], i32),
                "isprime_tuning_defaults": ([ctypes.POINTER(Tuning)], i32),
                "isprime_ctx_set_tuning": ([vp, ctypes.POINTER(Tuning)], i32),
                "isprime_ctx_stats": ([vp, ctypes.POINTER(_Stats)], i32),
                "isprime_u64": ([vp, vp, sz, vp], i32),
                "isprime_u64_ctx": ([vp, vp, vp, sz, vp], i32),
                "isprime_f64": ([vp, vp, sz, vp, vp], i32),
                "isprime_f64_ctx": ([vp, vp, vp, sz, vp, vp], i32),
                "isprime_f64_sync_status": ([vp, ctypes.POINTER(ctypes.c_ulonglong)], i32),
                "isprime_u64_host": ([vp, vp, vp, sz, vp], i32),
                "isprime_u64_scalar": ([vp, u64, ctypes.POINTER(ctypes.c_uint8)], i32),
                "isprime_range": ([vp, u64, u64, vp, vp], i32),
                "isprime_u64_batched": ([vp, ctypes.POINTER(ArrayDesc), sz, vp], i32),
                "isprime_autotune": ([vp, vp, vp, sz, i32, ctypes.c_char_p, ctypes.POINTER(Tuning)], i32),
                "isprime_tuning_format": ([ctypes.POINTER(Tuning), ctypes.c_char_p, sz], i32),
                "isprime_server_create": ([vp, sz, i32, ctypes.POINTER(vp)], i32),
                "isprime_server_submit": ([vp, vp, vp, sz, ctypes.POINTER(u64)], i32),
                "isprime_server_wait": ([vp, u64, i32], i32),
                "isprime_server_get_stats": ([vp, ctypes.POINTER(_ServerStats)], i32),
                "isprime_server_reset_stats": ([vp], i32),
                "isprime_server_destroy": ([vp], i32),
                "isprime_sieve_count": ([vp, ctypes.POINTER(u64)], i32),
                "isprime_timing_enable": ([vp, i32], i32),
                "isprime_timing_read": ([vp, ctypes.POINTER(_KTime), i32], i32),
                "isprime_timing_reset": ([vp], i32),
                "isprime_measure_int_rates": ([i32, ctypes.POINTER(_IntRates)], i32),
                "isprime_count_ops": ([vp, vp, vp, sz, ctypes.POINTER(_OpCounts)], i32),
                "isprime_debug_checks": ([i32, ctypes.POINTER(ctypes.c_uint32),
                                          ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_int)], i32),
                "isprime_plan_contiguous": ([u64, ctypes.c_uint32, vp], i32),
                "isprime_plan_batched": ([vp, sz, ctypes.c_uint32, vp, vp], i32),
                "isprime_u64_host_multi": ([vp, ctypes.c_uint32, vp, vp, sz], i32),
                "isprime_route_least_loaded": ([vp, ctypes.c_uint32,
                                                ctypes.POINTER(ctypes.c_uint32)], i32),
                "isprime_strerror": ([i32], ctypes.c_char_p),
                "isprime_last_error": ([], ctypes.c_char_p),
                "isprime_version": ([], i32),
            }
            for name, (args, res) in sigs.items():
                f = getattr(L, name)
                f.argtypes, f.restype = args, res
            _lib = L
    return _lib


def _check(status):
    if status != OK:
        L = lib()
        raise IsPrimeError(status, f"{L.isprime_strerror(status).decode()}: "
                                   f"{L.isprime_last_error().decode()}")


def _torch():
    import torch
    return torch


def _stream_handle(t, stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(t.device)
    return ctypes.c_void_p(stream.cuda_stream)


def _prep(t):
    """Contiguous CUDA tensor of 8-byte elements and its kind ('u64'|'f64')."""
    torch = _torch()
    if not t.is_cuda:
        raise ValueError("isprime expects a CUDA tensor (use isprime_host for host arrays)")
    if t.dtype == torch.float64:
        kind = "f64"
    elif t.dtype in (torch.int64, getattr(torch, "uint64", torch.int64)):
        kind = "u64"
    elif t.dtype in (torch.int32, torch.int16, torch.int8, torch.uint8, torch.bool):
        if t.dtype != torch.bool and t.numel() and bool((t < 0).any()):
            raise ValueError("negative integers are not valid isprime inputs")
        t = t.to(torch.int64)
        kind = "u64"
    else:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return t.contiguous(), kind


class Context:
    """A library context on one device: resident sieve, queues, tuning."""

    def __init__(self, device: int = 0, sieve_limit: int | None = None, _handle=None):
        self._owned = _handle is None
        if _handle is not None:
            self._h = _handle
        else:
            h = ctypes.c_void_p()
            _check(lib().isprime_ctx_create(device, SIEVE_DEFAULT if sieve_limit is None
                                            else sieve_limit, ctypes.byref(h)))
            self._h = h
        self.device = device

    @classmethod
    def default(cls, device: int = 0) -> "Context":
        h = ctypes.c_void_p()
        _check(lib().isprime_default_ctx(device, ctypes.byref(h)))
        return cls(device, _handle=h)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._owned and self._h:
            _check(lib().isprime_ctx_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- tuning / stats / timing
    @property
    def tuning(self) -> Tuning:
        t = Tuning()
        _check(lib().isprime_ctx_get_tuning(self._h, ctypes.byref(t)))
        return t

    def set_tuning(self, **kw):
        t = self.tuning
        for k, v in kw.items():
            setattr(t, k, v)
        _check(lib().isprime_ctx_set_tuning(self._h, ctypes.byref(t)))

    def stats(self) -> dict:
        s = _Stats()
        _check(lib().isprime_ctx_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def timing(self, on: bool = True):
        _check(lib().isprime_timing_enable(self._h, 1 if on else 0))

    def timing_read(self) -> dict:
        arr = (_KTime * len(KERNEL_NAMES))()
        _check(lib().isprime_timing_read(self._h, arr, len(KERNEL_NAMES)))
        return {name: (arr[i].total_ms, arr[i].launches) for i, name in enumerate(KERNEL_NAMES)}

    def timing_reset(self):
        _check(lib().isprime_timing_reset(self._h))

    def sieve_count(self) -> int:
        v = ctypes.c_uint64()
        _check(lib().isprime_sieve_count(self._h, ctypes.byref(v)))
        return int(v.value)

    # -- the operation
    def isprime(self, t, out=None, stream=None, invalid=None):
        """Elementwise primality of a CUDA tensor; uint8 tensor of t's shape.

        int64 / uint64 tensors are read as unsigned 64-bit values; float64
        tensors take the double path (invalid elements give 0 and, if
        `invalid` is a 1-element int64 CUDA tensor, are counted into it)."""
        torch = _torch()
        src, kind = _prep(t)
        if out is None:
            out = torch.empty(src.shape, dtype=torch.uint8, device=src.device)
        elif out.dtype != torch.uint8 or out.shape != src.shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous uint8 tensor of the input's shape")
        n = src.numel()
        if n == 0:
            return out
        sh = _stream_handle(src, stream)
        L = lib()
        if kind == "u64":
            _check(L.isprime_u64_ctx(self._h, src.data_ptr(), out.data_ptr(), n, sh))
        else:
            inv = None if invalid is None else ctypes.c_void_p(invalid.data_ptr())
            _check(L.isprime_f64_ctx(self._h, src.data_ptr(), out.data_ptr(), n, inv, sh))
        return out

    def count_ops(self, t) -> dict:
        """Executed Montgomery operations of the Miller-Rabin stages on one
        pass over the CUDA integer tensor t: {name: (warp issues, active
        lanes)} (see isprime_count_ops)."""
        torch = _torch()
        src, kind = _prep(t)
        if kind != "u64":
            raise TypeError("count_ops takes an integer tensor")
        out = torch.empty(src.numel(), dtype=torch.uint8, device=src.device)
        c = _OpCounts()
        _check(lib().isprime_count_ops(self._h, src.data_ptr(), out.data_ptr(), src.numel(),
                                       ctypes.byref(c)))
        res = {"elements": int(c.elements)}
        for k, _ in c._fields_[1:]:
            v = getattr(c, k)
            res[k] = (int(v[0]), int(v[1]))
        return res

    def f64_status(self) -> int:
        """Invalid double inputs (not integers in [0, 2^53]) seen by the
        context's double-path calls since the last status read; waits for
        those calls.  0 means ISPRIME_OK, more than 0 ISPRIME_EDOMAIN."""
        c = ctypes.c_ulonglong(0)
        st = lib().isprime_f64_sync_status(self._h, ctypes.byref(c))
        if st not in (OK, EDOMAIN):
            _check(st)
        return int(c.value)

    def autotune(self, sample, mode: str = "plain", cache_path: str | None = None) -> dict:
        """Times `sample` (a CUDA integer tensor) under candidate tunings and
        installs the fastest (see isprime_autotune)."""
        torch = _torch()
        src, kind = _prep(sample)
        out = torch.empty(src.numel(), dtype=torch.uint8, device=src.device)
        t = Tuning()
        m = {"plain": 0, "batched": 1}[mode]
        _check(lib().isprime_autotune(self._h, src.data_ptr(), out.data_ptr(), src.numel(), m,
                                      cache_path.encode() if cache_path else None, ctypes.byref(t)))
        return t.as_dict()

    def isprime_batched(self, tensors, outs=None, stream=None):
        """Classifies a list of CUDA tensors (any lengths) in one batched
        launch; returns the list of uint8 outputs."""
        torch = _torch()
        srcs = []
        for t in tensors:
            src, kind = _prep(t)
            if kind != "u64":
                raise TypeError("the batched form takes integer tensors")
            srcs.append(src)
        if outs is None:
            outs = [torch.empty(s.shape, dtype=torch.uint8, device=s.device) for s in srcs]
        descs = (ArrayDesc * max(len(srcs), 1))()
        for i, (s_, o) in enumerate(zip(srcs, outs)):
            descs[i].d_in = s_.data_ptr() if s_.numel() else None
            descs[i].d_out = o.data_ptr() if o.numel() else None
            descs[i].n = s_.numel()
        if srcs:
            sh = _stream_handle(srcs[0], stream)
            _check(lib().isprime_u64_batched(self._h, descs, len(srcs), sh))
        self._keep = srcs  # keep converted inputs alive until the stream runs them
        return outs

    def isprime_range(self, lo: int, count: int, out=None, stream=None):
        """uint8 CUDA tensor r with r[i] = isprime(lo + i), i < count."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        if out is None:
            out = torch.empty(count, dtype=torch.uint8, device=dev)
        if count:
            sh = ctypes.c_void_p((stream or torch.cuda.current_stream(dev)).cuda_stream)
            _check(lib().isprime_range(self._h, lo, count, out.data_ptr(), sh))
        return out

    def isprime_host(self, values, stream=None) -> np.ndarray:
        """End-to-end call on a host array (copies in, classifies, copies out)."""
        a = np.ascontiguousarray(values, dtype=np.uint64)
        out = np.empty(a.shape, dtype=np.uint8)
        if a.size:
            sh = ctypes.c_void_p(0 if stream is None else stream.cuda_stream)
            _check(lib().isprime_u64_host(self._h, a.ctypes.data, out.ctypes.data, a.size, sh))
        return out

    def isprime_scalar(self, value: int) -> bool:
        """isprime(value) for one Python int in [0, 2^64), one launch, synchronous."""
        if not 0 <= int(value) < 1 << 64:
            raise IsPrimeError(EINVAL, "value out of the uint64 range")
        r = ctypes.c_uint8()
        _check(lib().isprime_u64_scalar(self._h, int(value), ctypes.byref(r)))
        return bool(r.value)


class Server:
    """Continuous-batching server over a context (see isprime_server_create).

    submit() takes a host numpy array (uint64-compatible) and returns a
    ticket; the input and output arrays are kept alive until wait()."""

    def __init__(self, ctx: Context, mem_budget_bytes: int = 8 << 30, n_slots: int = 4):
        h = ctypes.c_void_p()
        _check(lib().isprime_server_create(ctx.handle, mem_budget_bytes, n_slots, ctypes.byref(h)))
        self._h = h
        self._ctx = ctx
        self._live: dict = {}

    def submit(self, values, out=None) -> int:
        a = np.ascontiguousarray(values)
        if a.dtype != np.uint64:
            a = a.astype(np.uint64)
        if out is None:
            out = np.empty(a.shape, dtype=np.uint8)
        t = ctypes.c_uint64()
        _check(lib().isprime_server_submit(self._h, a.ctypes.data if a.size else None,
                                           out.ctypes.data if out.size else None, a.size,
                                           ctypes.byref(t)))
        self._live[t.value] = (a, out)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> np.ndarray:
        _check(lib().isprime_server_wait(self._h, ticket, timeout_ms))
        return self._live.pop(ticket)[1]

    def stats(self) -> dict:
        s = _ServerStats()
        _check(lib().isprime_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def reset_stats(self):
        _check(lib().isprime_server_reset_stats(self._h))

    def close(self):
        if self._h:
            _check(lib().isprime_server_destroy(self._h))
            self._h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_defaults: dict = {}


def _default_ctx(device: int) -> Context:
    c = _defaults.get(device)
    if c is None:
        c = _defaults[device] = Context.default(device)
    return c


def isprime(t, out=None, stream=None, invalid=None):
    """Elementwise isprime of a CUDA tensor with the device's default context."""
    return _default_ctx(t.device.index or 0).isprime(t, out=out, stream=stream, invalid=invalid)


def isprime_host(values, device: int = 0) -> np.ndarray:
    return _default_ctx(device).isprime_host(values)


def default_tuning() -> dict:
    """The tuning a new context starts with (needs no GPU)."""
    t = Tuning()
    _check(lib().isprime_tuning_defaults(ctypes.byref(t)))
    return t.as_dict()


def isprime_scalar(value: int, device: int = 0) -> bool:
    return _default_ctx(device).isprime_scalar(value)


def debug_checks(reset: bool = True) -> dict:
    """Bounds-check record of the debug build (see isprime_debug_checks)."""
    s, v, c = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_int()
    _check(lib().isprime_debug_checks(1 if reset else 0, ctypes.byref(s), ctypes.byref(v),
                                      ctypes.byref(c)))
    return {"compiled": bool(c.value), "sites": int(s.value), "violations": int(v.value)}


def int_rates(device: int = 0) -> dict:
    r = _IntRates()
    _check(lib().isprime_measure_int_rates(device, ctypes.byref(r)))
    out = {k: getattr(r, k) for k, _ in r._fields_ if k != "mont_variant"}
    names = ["mul_128", "mul_word", "sqr_word", "sqr_128", "mul_128_ptxredc", "sqr_as_mul_128",
             "mul_fused", "sqr_fused", "mul_words_ptx", "sqr_words_ptx"]
    for i, nm in enumerate(names):
        out["mont_" + nm] = r.mont_variant[i]
    return out


# ------------------------------------------------ sharding a job across devices
# Host-only planning (no device is touched): which device takes which part.

def plan_contiguous(n: int, n_shards: int) -> np.ndarray:
    """Boundaries of n_shards contiguous ranges of n elements (sizes differ by
    at most one): shard s takes [begin[s], begin[s+1])."""
    begin = np.zeros(n_shards + 1 if n_shards > 0 else 1, dtype=np.uint64)
    _check(lib().isprime_plan_contiguous(n, n_shards, begin.ctypes.data))
    return begin


def plan_batched(sizes, n_shards: int) -> tuple[np.ndarray, np.ndarray]:
    """Whole arrays to n_shards, longest first to the least-loaded shard.
    Returns (owner per array, elements per shard)."""
    sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
    owner = np.zeros(sizes.size, dtype=np.uint32)
    load = np.zeros(max(n_shards, 1), dtype=np.uint64)
    _check(lib().isprime_plan_batched(sizes.ctypes.data if sizes.size else None, sizes.size,
                                      n_shards, owner.ctypes.data if sizes.size else None,
                                      load.ctypes.data))
    return owner, load


def isprime_host_multi(values, devices) -> np.ndarray:
    """A host array split over several devices (isprime_u64_host_multi)."""
    a = np.ascontiguousarray(values, dtype=np.uint64)
    out = np.empty(a.shape, dtype=np.uint8)
    d = np.ascontiguousarray(devices, dtype=np.int32)
    _check(lib().isprime_u64_host_multi(d.ctypes.data if d.size else None, d.size,
                                        a.ctypes.data if a.size else None,
                                        out.ctypes.data if a.size else None, a.size))
    return out


def route_least_loaded(outstanding) -> int:
    """The device with the least outstanding work (ties to the lower index)."""
    o = np.ascontiguousarray(outstanding, dtype=np.uint64)
    d = ctypes.c_uint32(0)
    _check(lib().isprime_route_least_loaded(o.ctypes.data if o.size else None, o.size,
                                            ctypes.byref(d)))
    return int(d.value)
