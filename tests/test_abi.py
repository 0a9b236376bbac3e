"""The C-ABI library builds, loads and exports every declared entry point.

CPU only: no call here touches a GPU (argument checks that fail before any
CUDA call, and metadata functions).
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2108_04791_gb300 as ipg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "isprime.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isprime_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    ipg.build()
    return ipg.lib()


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ("isprime_u64", "isprime_f64", "isprime_u64_ctx", "isprime_ctx_create",
                 "isprime_ctx_destroy", "isprime_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", ipg._build.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (isprime_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(L, n)


def test_header_compiles_as_c():
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c", HEADER],
                   check=True)


def test_metadata(L):
    assert L.isprime_version() >= 10000
    assert L.isprime_strerror(0) == b"ok"
    assert L.isprime_strerror(-1) == b"invalid argument"
    assert b"domain" in L.isprime_strerror(-4)


def test_argument_checks_without_gpu(L):
    buf = np.zeros(16, dtype=np.uint64)
    out = np.zeros(16, dtype=np.uint8)
    p_in, p_out = buf.ctypes.data, out.ctypes.data
    # n == 0 is a no-op
    assert L.isprime_u64(None, None, 0, None) == 0
    assert L.isprime_f64(None, None, 0, None, None) == 0
    # NULL with n > 0
    assert L.isprime_u64(None, p_out, 4, None) == ipg.EINVAL
    assert L.isprime_u64(p_in, None, 4, None) == ipg.EINVAL
    # misaligned input
    assert L.isprime_u64(p_in + 4, p_out, 4, None) == ipg.EINVAL
    assert b"aligned" in L.isprime_last_error()
    # overlapping output
    assert L.isprime_u64(p_in, p_in + 8, 4, None) == ipg.EINVAL
    assert b"overlap" in L.isprime_last_error()
    # NULL context
    assert L.isprime_u64_ctx(None, p_in, p_out, 4, None) == ipg.EINVAL
    assert L.isprime_u64_scalar(None, 5, ctypes.byref(ctypes.c_uint8())) == ipg.EINVAL
    assert L.isprime_u64_host(None, p_in, p_out, 4, None) == ipg.EINVAL
    assert L.isprime_ctx_destroy(None) == 0


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors have the sizes of the C structs in include/isprime.h."""
    src = tmp_path / "sizes.c"
    src.write_text('#include "isprime.h"\n#include <stdio.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(isprime_tuning),'
                   ' sizeof(isprime_stats), sizeof(isprime_kernel_time), sizeof(isprime_int_rates),'
                   ' sizeof(isprime_array)); printf("%zu\\n", sizeof(isprime_server_stats));'
                   ' printf("%zu\\n", sizeof(isprime_op_counts)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                            check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(ipg.Tuning), ctypes.sizeof(ipg._Stats), ctypes.sizeof(ipg._KTime),
                     ctypes.sizeof(ipg._IntRates), ctypes.sizeof(ipg.ArrayDesc),
                     ctypes.sizeof(ipg._ServerStats), ctypes.sizeof(ipg._OpCounts)]


def test_tuning_struct_matches_the_binding(L):
    """The Python binding's Tuning mirrors isprime_tuning field by field (names
    and order, all uint32_t), and the defaults read back through
    isprime_tuning_defaults land in the right fields."""
    src = open(HEADER).read()
    body = src[src.index("typedef struct"):src.index("} isprime_tuning;")]
    body = body[body.rindex("typedef struct"):]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(uint32_t|uint64_t|int)\s+([a-z0-9_]+)\s*;", body)
    assert fields and all(t == "uint32_t" for t, _ in fields)
    assert [n for _, n in fields] == [n for n, _ in ipg.Tuning._fields_]
    d = ipg.default_tuning()
    assert d["chunk_log2"] == 24 and d["td_primes"] == 15 and d["td2_groups"] == 16
    assert d["rest_ilp"] == 2 and d["td_fold"] == 3 and d["mont_impl"] == 9
    assert d["serve_long_log2"] == 24 and d["host_chunk_log2"] == 22 and d["inplace_max_log2"] == 0
