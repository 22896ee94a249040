"""The product path stands alone (CPU only).

The package must never reach the CPU oracle (test infrastructure) and must
fail loudly, not fall back to another implementation, when libfht.so is
missing.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2411_07351_gb300")

MODULES = ["paper_2411_07351_gb300", "paper_2411_07351_gb300._capi", "paper_2411_07351_gb300.fht",
           "paper_2411_07351_gb300.autograd", "paper_2411_07351_gb300.batch", "paper_2411_07351_gb300.serve",
           "paper_2411_07351_gb300.tune", "paper_2411_07351_gb300.experiments",
           "paper_2411_07351_gb300.parallel", "paper_2411_07351_gb300.inputs"]


def test_package_sources_never_name_the_oracle_module():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".cpp", ".hpp", ".h")):
                continue
            with open(os.path.join(dirpath, f)) as fh:
                for ln, line in enumerate(fh, 1):
                    s = line.strip()
                    assert not (s.startswith(("import oracle", "from oracle")) or "fht_oracle" in s
                                or "orc_" in s), f"{f}:{ln} reaches the oracle"


def test_importing_the_package_loads_no_oracle():
    code = ("import sys, importlib\n"
            f"for m in {MODULES!r}: importlib.import_module(m)\n"
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
            "assert not bad, bad\n"
            "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]


def test_missing_library_fails_loudly(tmp_path):
    code = ("import sys\n"
            "from paper_2411_07351_gb300 import _capi\n"
            "try:\n"
            f"    _capi.load({str(tmp_path / 'libfht.so')!r})\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    sys.exit('loaded a library that does not exist')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "raised:" in r.stdout, r.stdout + r.stderr


@pytest.mark.parametrize("name", ["fht_forward", "fht_adjoint", "fht_submit"])
def test_binding_calls_the_c_abi(name):
    # the Python layer marshals arguments only: each compute call goes through libfht.so
    src = "".join(open(os.path.join(PKG, f)).read() for f in ("fht.py", "batch.py", "_capi.py"))
    assert name in src
