"""The C-ABI library builds, loads and exports what include/gcc_gb300.h
declares; the ctypes binding agrees with the C compiler on struct layouts.
No GPU needed (no compute call is made)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2406_10158_gb300 import build as B
from paper_2406_10158_gb300 import engine as eng

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for h in os.listdir(HEADER_DIR):
        if h.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*[\w\s\*]+?\b(gcc_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    B.build()
    return ctypes.CDLL(B.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"gcc_db_create", "gcc_load_table", "gcc_txn_batch_submit", "gcc_batch_wait"} <= names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert declared_functions() == set(eng.SIGNATURES)


def test_binding_loads_and_reports_errors(lib):
    eng.load()
    # argument validation happens before any device call
    with pytest.raises(eng.GCCError) as e:
        eng.gcc_db_create(eng.DbDesc(schema=7))
    assert "schema" in str(e.value)
    p = eng.params(lanes_per_txn=8)
    assert p.lanes_per_txn == 8 and p.max_attempts == 1 << 24


def test_struct_layouts_match_c(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    prog = tmp_path / "layout.c"
    structs = {"gcc_db_desc": eng.DbDesc, "gcc_exec_params": eng.ExecParams,
               "gcc_batch_stats": eng.BatchStats, "gcc_stage_times": eng.StageTimes,
               "gcc_tune_space": eng.TuneSpace, "gcc_tune_report": eng.TuneReport,
               "gcc_memory_probe": eng.MemoryProbe,
               "gcc_multi_batch": eng.MultiBatch, "gcc_server_lane": eng.ServerLane,
               "gcc_completion": eng.Completion}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gcc_gb300.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    for cname in ("gcc_txn", "gcc_op", "gcc_operand", "gcc_txn_result"):
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", HEADER_DIR, "-o", str(exe), str(prog)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)
    from paper_2406_10158_gb300 import workload as wl
    assert int(out["gcc_txn"]) == wl.TXN_DTYPE.itemsize
    assert int(out["gcc_op"]) == wl.OP_DTYPE.itemsize
    assert int(out["gcc_operand"]) == 16
    assert int(out["gcc_txn_result"]) == wl.RESULT_DTYPE.itemsize
