"""The debug build: the library compiled with IP_DEBUG_CHECKS bounds-checks
every queue append, queue read and output store of its kernels and records
violations in device words (no trap).  This test builds it (on the machine
that runs the test), runs the parity cases of tests/debug_check_cases.py
under it in a child process, and asserts that every case equals the oracle
and that no check fired."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

import paper_2108_04791_gb300._build as build  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_runs_the_parity_cases_with_every_check_clear():
    path = build.build(debug=True)
    env = dict(os.environ, ISPRIME_GB300_LIB=path)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_check_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert res["after"]["compiled"] is True
    assert res["cases"] >= 20 and res["mismatches"] == [], res
    assert res["after"]["sites"] == 0 and res["after"]["violations"] == 0, res


def test_production_build_has_the_checks_compiled_out():
    import paper_2108_04791_gb300 as ipg
    rec = ipg.debug_checks(reset=False)
    assert rec == {"compiled": False, "sites": 0, "violations": 0}
