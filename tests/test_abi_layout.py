"""The Python binding and include/fht.h agree (CPU only).

A small C program compiled with gcc against the header prints the size and
every field offset of the structs the binding mirrors, and the value of every
constant it restates; the ctypes structures, the numpy job layout and the
Python constants must match them exactly.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2411_07351_gb300 import _capi as C
from paper_2411_07351_gb300 import batch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "fht_tuning_t": C.fht_tuning_t,
    "fht_plan_info_t": C.fht_plan_info_t,
    "fht_job": C.fht_job,
}

CONSTANTS = ["FHT_OK", "FHT_ERR_INVALID", "FHT_ERR_NOMEM", "FHT_ERR_CUDA", "FHT_ERR_TIMEOUT", "FHT_ERR_BUSY",
             "FHT_ERR_UNSUPPORTED", "FHT_ERR_DEVICE", "FHT_U8_I32", "FHT_I32_I32", "FHT_F32_F32", "FHT_F64_F64",
             "FHT_Q0", "FHT_Q1", "FHT_Q2", "FHT_Q3", "FHT_QALL", "FHT_CYCLIC", "FHT_EXTENDED", "FHT_SPLIT_T",
             "FHT_SPLIT_S", "FHT_JOB_WITHHOLD_DEPENDENCY", "FHT_TABLE_QUADS", "FHT_TABLE_FUSED", "FHT_TABLE_OPS",
             "FHT_TABLE_ROWS", "FHT_TABLE_PASS_BEGIN", "FHT_TABLE_BAND_ITEMS", "FHT_TABLE_SPINE_ROWS",
             "FHT_TABLE_SPINE_TERMS", "FHT_TABLE_SPINE_BEGIN", "FHT_TABLE_ADJ_ROWS", "FHT_TABLE_ADJ_TERMS",
             "FHT_TABLE_ADJ_BEGIN", "FHT_TABLE_ADJ_PTR", "FHT_TABLE_ADJ_OPS"]


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fht.h"', "int main(void) {"]
    for name, st in STRUCTS.items():
        lines.append(f'  printf("size {name} %zu\\n", sizeof({name}));')
        for fname, _ in st._fields_:
            lines.append(f'  printf("off {name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    for c in CONSTANTS:
        lines.append(f'  printf("const {c} %lld\\n", (long long)({c}));')
    lines += ["  return 0;", "}"]
    src = d / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "probe"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        kind, key, val = ln.split()
        got[(kind, key)] = int(val)
    return got


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_layout_matches_header(layout, name):
    st = STRUCTS[name]
    assert ctypes.sizeof(st) == layout[("size", name)]
    for fname, _ in st._fields_:
        assert getattr(st, fname).offset == layout[("off", f"{name}.{fname}")], f"{name}.{fname}"


def test_numpy_job_layout_matches_header(layout):
    dt = batch._JOB_DTYPE
    assert dt.itemsize == layout[("size", "fht_job")]
    for fname in dt.names:
        assert dt.fields[fname][1] == layout[("off", f"fht_job.{fname}")], fname


def test_constants_match_header(layout):
    for c in CONSTANTS:
        assert getattr(C, c) == layout[("const", c)], c
