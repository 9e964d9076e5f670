"""Argument checks of the C ABI, exercised on the CPU.

Every entry point validates its arguments before it touches the CUDA runtime
and reports a bad one with the status the header documents and a message
from gcc_last_error().  These calls make no device call, so they run without
a GPU; the library is the one the GPU tests use.
"""
import ctypes
import os
import shutil

import pytest

from paper_2406_10158_gb300 import build as B
from paper_2406_10158_gb300 import engine as eng

OK, INVALID, CAPACITY = 0, 1, 6
KV, OE = 0, 1


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    B.build()
    return eng.load()


def last_error(lib) -> str:
    return lib.gcc_last_error().decode()


def expect(lib, rc, status, words=()):
    assert rc == status, (rc, status, last_error(lib))
    msg = last_error(lib)
    for w in words:
        assert w in msg, (w, msg)


def kv_desc(**kw):
    d = eng.DbDesc(schema=KV, field_bytes=8, n_records=1024, n_fields=4, max_ops_per_txn=16,
                   max_batch_txns=1024, max_batch_ops=16384)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def oe_desc(**kw):
    d = eng.DbDesc(schema=OE, n_warehouses=2, order_cap=4096, max_ops_per_txn=33,
                   max_batch_txns=1024, max_batch_ops=33 * 1024)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("desc,words", [
    (kv_desc(schema=7), ["schema"]),
    (kv_desc(field_bytes=12), ["field_bytes"]),
    (kv_desc(n_records=0), ["n_records"]),
    (kv_desc(n_records=(1 << 31) + 1), ["n_records"]),
    (kv_desc(n_fields=0), ["n_fields"]),
    (kv_desc(n_fields=256), ["n_fields"]),
    (kv_desc(max_ops_per_txn=0), ["max_ops_per_txn"]),
    (kv_desc(max_ops_per_txn=65), ["max_ops_per_txn"]),
    (kv_desc(max_batch_txns=0), ["max_batch_txns"]),
    (kv_desc(max_batch_txns=(1 << 31) + 1), ["max_batch_txns"]),
    (kv_desc(max_batch_ops=0), ["max_batch_ops"]),
    (kv_desc(max_batch_ops=1 << 32), ["max_batch_ops"]),
    (oe_desc(n_warehouses=0), ["n_warehouses"]),
    (oe_desc(n_warehouses=1025), ["n_warehouses"]),
    (oe_desc(order_cap=2999), ["order_cap"]),
    (oe_desc(order_cap=(1 << 24) + 1), ["order_cap"]),
])
def test_db_create_rejects_each_bad_field(lib, desc, words):
    h = ctypes.c_void_p(123)
    expect(lib, lib.gcc_db_create(ctypes.byref(desc), ctypes.byref(h)), INVALID, words)
    assert h.value is None                     # *out cleared on failure


def test_null_handles(lib):
    expect(lib, lib.gcc_db_create(None, None), INVALID, ["null"])
    expect(lib, lib.gcc_default_params(None), INVALID, ["null"])
    assert lib.gcc_db_destroy(None) == OK
    assert lib.gcc_table_count(None) == 0 and lib.gcc_table_bytes(None, 0) == 0
    buf = ctypes.create_string_buffer(16)
    expect(lib, lib.gcc_load_table(None, 0, buf, 16, 0), INVALID, ["null"])
    expect(lib, lib.gcc_db_read_table(None, 0, buf, 16, 0), INVALID, ["null"])
    expect(lib, lib.gcc_init_table_seeded(None, 0, 1), INVALID, ["null"])
    expect(lib, lib.gcc_execute(None, 0, None, 0, None, None, 0, None, None, None, None),
           INVALID, ["null database"])
    expect(lib, lib.gcc_last_stats(None, None), INVALID, ["null"])
    n = ctypes.c_uint32(0)
    expect(lib, lib.gcc_stage_history(None, 0, None, ctypes.byref(n)), INVALID, ["null"])
    out = ctypes.c_void_p(0)
    expect(lib, lib.gcc_txn_batch_submit(None, 0, None, 0, None, None, 0, 0, None, None,
                                         ctypes.byref(out)), INVALID, ["null"])
    expect(lib, lib.gcc_batch_wait(None, 0, None, None, None, 0), INVALID, ["null"])
    assert lib.gcc_batch_free(None) == OK
    best = eng.ExecParams()
    expect(lib, lib.gcc_autotune(None, 0, None, 0, None, None, 0, None, None, None,
                                 ctypes.byref(best), None, None), INVALID, ["null"])
    expect(lib, lib.gcc_probe_memory(0, None), INVALID, ["NULL"])


def test_multi_plan_checks(lib):
    out = ctypes.c_void_p(0)
    expect(lib, lib.gcc_multi_plan_create(0, None, 0, None, ctypes.byref(out)), INVALID)
    many = (eng.MultiBatch * 257)()
    expect(lib, lib.gcc_multi_plan_create(2, many, 257, None, ctypes.byref(out)), CAPACITY,
           ["256"])
    one = (eng.MultiBatch * 1)()
    expect(lib, lib.gcc_multi_plan_create(7, one, 1, None, ctypes.byref(out)), INVALID,
           ["unknown scheme"])
    bad = eng.ExecParams(lanes_per_txn=3)
    expect(lib, lib.gcc_multi_plan_create(2, one, 1, ctypes.byref(bad), ctypes.byref(out)),
           INVALID, ["lanes_per_txn"])
    expect(lib, lib.gcc_multi_plan_create(2, one, 1, None, ctypes.byref(out)), INVALID,
           ["key-value database"])
    assert out.value is None
    expect(lib, lib.gcc_multi_launch(None, 0, None), INVALID, ["null"])
    expect(lib, lib.gcc_multi_stats(None, 0, None), INVALID)
    assert lib.gcc_multi_plan_destroy(None) == OK


@pytest.mark.parametrize("field,value,words", [
    ("lanes_per_txn", 3, ["lanes_per_txn"]),
    ("lanes_per_txn", 64, ["lanes_per_txn"]),
    ("warps_per_block", 33, ["warps_per_block"]),
    ("collapse", 3, ["collapse"]),
    ("retry_queue", 3, ["retry_queue"]),
    ("det_dataflow", 3, ["det_dataflow"]),
])
def test_exec_params_are_validated(lib, field, value, words):
    """validate_params runs before a plan looks at its databases."""
    p = eng.ExecParams()
    setattr(p, field, value)
    one = (eng.MultiBatch * 1)()
    out = ctypes.c_void_p(0)
    expect(lib, lib.gcc_multi_plan_create(0, one, 1, ctypes.byref(p), ctypes.byref(out)),
           INVALID, words)


def test_server_checks(lib):
    out = ctypes.c_void_p(0)
    expect(lib, lib.gcc_server_create(None, 0, None, ctypes.byref(out)), INVALID, ["no lanes"])
    lanes = (eng.ServerLane * 1)()
    expect(lib, lib.gcc_server_create(lanes, 1, None, ctypes.byref(out)), INVALID,
           ["bad database"])
    assert out.value is None
    rid = ctypes.c_uint64(0)
    expect(lib, lib.gcc_server_enqueue(None, 0, None, None, None, 0, ctypes.byref(rid)), INVALID)
    expect(lib, lib.gcc_server_pump(None), INVALID, ["null"])
    expect(lib, lib.gcc_server_drain(None), INVALID, ["null"])
    n = ctypes.c_uint32(0)
    expect(lib, lib.gcc_server_completions(None, None, None, 0, 0, ctypes.byref(n)), INVALID)
    expect(lib, lib.gcc_server_run_trace(None, 0, None, None, None, None, None, None, None),
           INVALID)
    expect(lib, lib.gcc_server_lane_totals(None, 0, None, None, None), INVALID)
    assert lib.gcc_server_destroy(None) == OK
    t0 = lib.gcc_server_now_ns()
    assert lib.gcc_server_now_ns() >= t0 > 0


def test_noalloc_checks(lib):
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)

    def call(n_records=64, n_fields=2, field_bytes=8, n_txns=1, n_ops=1, max_ops=4, table=p):
        return lib.gcc_det_execute_noalloc(table, n_records, n_fields, field_bytes, p, n_txns,
                                           p, p, n_ops, max_ops, p, p, None)

    expect(lib, call(n_records=0), CAPACITY, ["65536"])
    expect(lib, call(n_records=65537), CAPACITY, ["65536"])
    expect(lib, call(n_ops=65537), CAPACITY, ["65536"])
    expect(lib, call(field_bytes=12), INVALID, ["field_bytes"])
    expect(lib, call(n_fields=0), INVALID, ["n_fields"])
    expect(lib, call(n_fields=256), INVALID, ["n_fields"])
    expect(lib, call(max_ops=0), INVALID, ["max_ops_per_txn"])
    expect(lib, call(max_ops=65), INVALID, ["max_ops_per_txn"])
    expect(lib, call(table=None), INVALID, ["null"])


def test_binding_raises_with_the_status(lib):
    with pytest.raises(eng.GCCError) as e:
        eng.gcc_db_create(kv_desc(field_bytes=4))
    assert e.value.status == INVALID and "field_bytes" in str(e.value)
