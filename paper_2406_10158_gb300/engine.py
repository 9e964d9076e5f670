"""Thin ctypes binding of the engine's C ABI (include/gcc_gb300.h).

Argument marshalling only: every step of a batch runs in the CUDA library.
The module-level ``gcc_*`` functions mirror the C entry points one to one;
``Database`` and ``Batch`` wrap them for numpy inputs (host path) and torch
CUDA tensors (device-resident path).  Loading fails loudly when the compiled
library is absent -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import workload as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgcc_gb300.so")

SCHEMES = {"2pl": 0, "no_wait_2pl": 0, "to": 1, "occ": 2, "det": 3, "tictoc": 4,
           "2pl_wd": 5, "wait_die": 5, "mvcc": 6}
SCHEME_NAMES = {0: "2pl", 1: "to", 2: "occ", 3: "det", 4: "tictoc", 5: "2pl_wd", 6: "mvcc"}
SCHEMA_KV, SCHEMA_ORDER_ENTRY = 0, 1
TXN_PENDING, TXN_COMMITTED, TXN_TIMEOUT, TXN_INVALID = 0, 1, 2, 3
STATUS = {0: "ok", 1: "invalid", 2: "cuda", 3: "timeout", 4: "nomem", 5: "device", 6: "capacity"}
DEVERR = {0x1: "wait_budget", 0x2: "deadline", 0x4: "ts_overflow", 0x8: "attempts",
          0x10: "invalid", 0x20: "insert"}
WAIT_FOREVER = (1 << 64) - 1


class DbDesc(ctypes.Structure):
    _fields_ = [("schema", ctypes.c_uint32), ("field_bytes", ctypes.c_uint32),
                ("n_records", ctypes.c_uint64), ("n_fields", ctypes.c_uint32),
                ("n_warehouses", ctypes.c_uint32), ("order_cap", ctypes.c_uint32),
                ("max_ops_per_txn", ctypes.c_uint32), ("max_batch_txns", ctypes.c_uint64),
                ("max_batch_ops", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class ExecParams(ctypes.Structure):
    _fields_ = [("lanes_per_txn", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("collapse", ctypes.c_uint32),
                ("backoff_base_ns", ctypes.c_uint32), ("backoff_cap_ns", ctypes.c_uint32),
                ("max_attempts", ctypes.c_uint32), ("read_retries", ctypes.c_uint32),
                ("wait_budget_ns", ctypes.c_uint64), ("deadline_ns", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("inject_abort_ppm", ctypes.c_uint32),
                ("immediate_restart", ctypes.c_uint32), ("det_dataflow", ctypes.c_uint32),
                ("retry_queue", ctypes.c_uint32), ("queue_turn_ns", ctypes.c_uint32),
                ("queue_width", ctypes.c_uint32), ("queue_after", ctypes.c_uint32),
                ("group_commit", ctypes.c_uint32), ("group_min_writes", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_txns", ctypes.c_uint64), ("committed", ctypes.c_uint64),
                ("aborts", ctypes.c_uint64), ("timeouts", ctypes.c_uint64),
                ("invalid", ctypes.c_uint64), ("max_attempts", ctypes.c_uint64),
                ("device_error", ctypes.c_uint32), ("scheme", ctypes.c_uint32),
                ("elapsed_ms", ctypes.c_double), ("prep_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("order_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_uint32), ("grid_blocks", ctypes.c_uint32),
                ("atomics", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["scheme"] = SCHEME_NAMES.get(d["scheme"], d["scheme"])
        d["abort_rate"] = d["aborts"] / d["committed"] if d["committed"] else float("nan")
        d["errors"] = [n for b, n in DEVERR.items() if d["device_error"] & b]
        return d


class StageTimes(ctypes.Structure):
    _fields_ = [("prep_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("order_ms", ctypes.c_double), ("scheme", ctypes.c_uint32),
                ("n_txns", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32),
                ("grid_blocks", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneSpace(ctypes.Structure):
    _fields_ = [("n_lanes", ctypes.c_uint32), ("lanes", ctypes.c_uint32 * 6),
                ("n_warps", ctypes.c_uint32), ("warps", ctypes.c_uint32 * 8),
                ("n_caps", ctypes.c_uint32), ("caps", ctypes.c_uint32 * 4),
                ("steps", ctypes.c_uint32), ("warmup", ctypes.c_uint32),
                ("point_deadline_ns", ctypes.c_uint64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("points", ctypes.c_uint32), ("best_index", ctypes.c_uint32),
                ("best_txn_per_s", ctypes.c_double), ("default_txn_per_s", ctypes.c_double)]


def tune_space(lanes=(), warps=(), caps=(), steps=0, warmup=0, point_deadline_ns=0) -> TuneSpace:
    sp = TuneSpace()
    sp.n_lanes, sp.n_warps, sp.n_caps = len(lanes), len(warps), len(caps)
    for i, v in enumerate(lanes):
        sp.lanes[i] = v
    for i, v in enumerate(warps):
        sp.warps[i] = v
    for i, v in enumerate(caps):
        sp.caps[i] = v
    sp.steps, sp.warmup, sp.point_deadline_ns = steps, warmup, point_deadline_ns
    return sp


class MultiBatch(ctypes.Structure):
    _fields_ = [("db", ctypes.c_void_p), ("d_txns", ctypes.c_void_p), ("n_txns", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("d_ops", ctypes.c_void_p),
                ("d_operands", ctypes.c_void_p), ("n_ops", ctypes.c_uint64),
                ("d_results", ctypes.c_void_p), ("d_reads", ctypes.c_void_p)]


class ServerLane(ctypes.Structure):
    _fields_ = [("db", ctypes.c_void_p), ("scheme", ctypes.c_uint32),
                ("max_batch_txns", ctypes.c_uint32), ("write_budget_bytes", ctypes.c_uint64),
                ("max_delay_ns", ctypes.c_uint64), ("depth", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class Completion(ctypes.Structure):
    _fields_ = [("request", ctypes.c_uint64), ("lane", ctypes.c_uint32), ("status", ctypes.c_uint32),
                ("batch_seq", ctypes.c_uint64), ("commit_order", ctypes.c_uint64),
                ("arrival_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64)]


class MemoryProbe(ctypes.Structure):
    _fields_ = [("hbm_load_ns", ctypes.c_double), ("l2_load_ns", ctypes.c_double),
                ("l2_load_acquire_ns", ctypes.c_double), ("l2_atomic_ns", ctypes.c_double),
                ("l2_cas_ns", ctypes.c_double), ("gather32_gbs", ctypes.c_double),
                ("cas_distinct_gops", ctypes.c_double), ("add_same_gops", ctypes.c_double),
                ("lock_handoff_ns", ctypes.c_double), ("occ_cycle_ns", ctypes.c_double),
                ("occ_cycle_busy_ns", ctypes.c_double),
                ("sm_count", ctypes.c_uint32), ("contenders", ctypes.c_uint32),
                ("lock_best_contenders", ctypes.c_uint32), ("occ_best_contenders", ctypes.c_uint32),
                ("fence_ns", ctypes.c_double), ("atomic_acq_rel_ns", ctypes.c_double),
                ("occ_link_ns", ctypes.c_double), ("occ_link_max_ns", ctypes.c_double),
                ("gather32_by_inflight_gbs", ctypes.c_double * 3),
                ("gather32_best_inflight", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


COMPLETION_DTYPE = np.dtype([("request", "<u8"), ("lane", "<u4"), ("status", "<u4"),
                             ("batch_seq", "<u8"), ("commit_order", "<u8"),
                             ("arrival_ns", "<u8"), ("done_ns", "<u8")])


class GCCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
P = ctypes.c_void_p

# name -> (restype, argtypes); mirrors include/gcc_gb300.h
SIGNATURES = {
    "gcc_db_create": (ctypes.c_int, [ctypes.POINTER(DbDesc), ctypes.POINTER(P)]),
    "gcc_db_destroy": (ctypes.c_int, [P]),
    "gcc_table_count": (ctypes.c_uint32, [P]),
    "gcc_table_bytes": (ctypes.c_uint64, [P, ctypes.c_uint32]),
    "gcc_load_table": (ctypes.c_int, [P, ctypes.c_uint32, P, ctypes.c_uint64, ctypes.c_int]),
    "gcc_db_read_table": (ctypes.c_int, [P, ctypes.c_uint32, P, ctypes.c_uint64, ctypes.c_int]),
    "gcc_init_table_seeded": (ctypes.c_int, [P, ctypes.c_uint32, ctypes.c_uint64]),
    "gcc_default_params": (ctypes.c_int, [ctypes.POINTER(ExecParams)]),
    "gcc_txn_batch_submit": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_uint32, P, P,
                                            ctypes.c_uint64, ctypes.c_int,
                                            ctypes.POINTER(ExecParams), P, ctypes.POINTER(P)]),
    "gcc_batch_wait": (ctypes.c_int, [P, ctypes.c_uint64, P, P, ctypes.POINTER(BatchStats),
                                      ctypes.c_int]),
    "gcc_batch_free": (ctypes.c_int, [P]),
    "gcc_execute": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_uint32, P, P, ctypes.c_uint64,
                                   ctypes.POINTER(ExecParams), P, P, P]),
    "gcc_last_stats": (ctypes.c_int, [P, ctypes.POINTER(BatchStats)]),
    "gcc_stage_history": (ctypes.c_int, [P, ctypes.c_uint32, P, ctypes.POINTER(ctypes.c_uint32)]),
    "gcc_multi_plan_create": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_uint32,
                                             ctypes.POINTER(ExecParams), ctypes.POINTER(P)]),
    "gcc_multi_launch": (ctypes.c_int, [P, ctypes.c_int, P]),
    "gcc_multi_stats": (ctypes.c_int, [P, ctypes.c_uint32, ctypes.POINTER(BatchStats)]),
    "gcc_multi_plan_destroy": (ctypes.c_int, [P]),
    "gcc_server_create": (ctypes.c_int, [P, ctypes.c_uint32, ctypes.POINTER(ExecParams),
                                         ctypes.POINTER(P)]),
    "gcc_server_enqueue": (ctypes.c_int, [P, ctypes.c_uint32, P, P, P, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "gcc_server_pump": (ctypes.c_int, [P]),
    "gcc_server_drain": (ctypes.c_int, [P]),
    "gcc_server_completions": (ctypes.c_int, [P, P, P, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.POINTER(ctypes.c_uint32)]),
    "gcc_server_run_trace": (ctypes.c_int, [P, ctypes.c_uint32, P, P, P, P, P, P, P]),
    "gcc_server_now_ns": (ctypes.c_uint64, []),
    "gcc_server_lane_totals": (ctypes.c_int, [P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64)]),
    "gcc_server_destroy": (ctypes.c_int, [P]),
    "gcc_autotune": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_uint32, P, P, ctypes.c_uint64,
                                    P, P, ctypes.POINTER(TuneSpace), ctypes.POINTER(ExecParams),
                                    ctypes.POINTER(TuneReport), P]),
    "gcc_det_execute_noalloc": (ctypes.c_int, [P, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_uint32, P, ctypes.c_uint32, P, P,
                                               ctypes.c_uint32, ctypes.c_uint32, P, P, P]),
    "gcc_probe_memory": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(MemoryProbe)]),
    "gcc_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load the compiled engine; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA engine library not found at {path}; build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise GCCError(status, load().gcc_last_error().decode(errors="replace"))


def params(**kw) -> ExecParams:
    """Execution parameters: the library defaults overridden by ``kw``."""
    p = ExecParams()
    _check(load().gcc_default_params(ctypes.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, int(v))
    return p


def _scheme(s) -> int:
    return SCHEMES[s.lower()] if isinstance(s, str) else int(s)


def _host_ptr(a: np.ndarray) -> int:
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _tensor_ptr(t) -> int:
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def gcc_db_create(desc: DbDesc) -> int:
    h = P()
    _check(load().gcc_db_create(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def gcc_db_destroy(db: int):
    _check(load().gcc_db_destroy(db))


def gcc_load_table(db: int, table_id: int, src_ptr: int, nbytes: int, on_device: bool):
    _check(load().gcc_load_table(db, table_id, src_ptr, nbytes, int(on_device)))


def gcc_init_table_seeded(db: int, table_id: int, seed: int):
    _check(load().gcc_init_table_seeded(db, table_id, seed & ((1 << 64) - 1)))


def gcc_db_read_table(db: int, table_id: int, dst_ptr: int, nbytes: int, on_device: bool):
    _check(load().gcc_db_read_table(db, table_id, dst_ptr, nbytes, int(on_device)))


def gcc_txn_batch_submit(db: int, scheme, txns_ptr: int, n_txns: int, ops_ptr: int,
                         operands_ptr: int, n_ops: int, inputs_on_device: bool,
                         p: Optional[ExecParams] = None, stream: int = 0) -> int:
    h = P()
    _check(load().gcc_txn_batch_submit(db, _scheme(scheme), txns_ptr, n_txns, ops_ptr,
                                       operands_ptr, n_ops, int(inputs_on_device),
                                       ctypes.byref(p) if p is not None else None,
                                       stream or None, ctypes.byref(h)))
    return h.value


def gcc_batch_wait(batch: int, timeout_ns: int, results_ptr, reads_ptr,
                   outputs_on_device: bool = False, check: bool = True) -> dict:
    st = BatchStats()
    rc = load().gcc_batch_wait(batch, timeout_ns, results_ptr, reads_ptr, ctypes.byref(st),
                               int(outputs_on_device))
    if check and rc not in (0, 5):
        _check(rc)
    d = st.as_dict()
    d["status"] = STATUS.get(rc, rc)
    return d


def gcc_batch_free(batch: int):
    _check(load().gcc_batch_free(batch))


def gcc_execute(db: int, scheme, txns_ptr: int, n_txns: int, ops_ptr: int, operands_ptr: int,
                n_ops: int, p: Optional[ExecParams], results_ptr: int, reads_ptr: int,
                stream: int = 0):
    _check(load().gcc_execute(db, _scheme(scheme), txns_ptr, n_txns, ops_ptr, operands_ptr,
                              n_ops, ctypes.byref(p) if p is not None else None, results_ptr,
                              reads_ptr, stream or None))


def gcc_last_stats(db: int) -> dict:
    st = BatchStats()
    _check(load().gcc_last_stats(db, ctypes.byref(st)))
    return st.as_dict()


def gcc_stage_history(db: int, max_entries: int = 256) -> list:
    arr = (StageTimes * max(1, max_entries))()
    n = ctypes.c_uint32(0)
    _check(load().gcc_stage_history(db, max_entries, arr, ctypes.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def gcc_autotune(db: int, scheme, txns_ptr: int, n_txns: int, ops_ptr: int, operands_ptr: int,
                 n_ops: int, results_ptr: int, reads_ptr: int, space: Optional[TuneSpace] = None,
                 stream: int = 0):
    """Returns (best ExecParams, report dict)."""
    best = ExecParams()
    rep = TuneReport()
    _check(load().gcc_autotune(db, _scheme(scheme), txns_ptr, n_txns, ops_ptr, operands_ptr,
                               n_ops, results_ptr, reads_ptr,
                               ctypes.byref(space) if space is not None else None,
                               ctypes.byref(best), ctypes.byref(rep), stream or None))
    return best, {k: getattr(rep, k) for k, _ in rep._fields_}


def gcc_probe_memory(device: int = 0) -> dict:
    """Memory-system figures of `device` (latencies in ns, rates per second)."""
    m = MemoryProbe()
    _check(load().gcc_probe_memory(device, ctypes.byref(m)))
    out = {}
    for k, _ in m._fields_:
        if k == "reserved":
            continue
        v = getattr(m, k)
        out[k] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def gcc_multi_plan_create(scheme, batches, p: Optional[ExecParams] = None) -> int:
    arr = (MultiBatch * len(batches))(*batches)
    h = P()
    _check(load().gcc_multi_plan_create(_scheme(scheme), arr, len(batches),
                                        ctypes.byref(p) if p is not None else None,
                                        ctypes.byref(h)))
    return h.value


def gcc_multi_launch(plan: int, use_graph: bool = True, stream: int = 0):
    _check(load().gcc_multi_launch(plan, int(use_graph), stream or None))


def gcc_multi_stats(plan: int, i: int) -> dict:
    st = BatchStats()
    _check(load().gcc_multi_stats(plan, i, ctypes.byref(st)))
    return st.as_dict()


def gcc_multi_plan_destroy(plan: int):
    _check(load().gcc_multi_plan_destroy(plan))


def gcc_last_error() -> str:
    return load().gcc_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------
# object wrappers
# ---------------------------------------------------------------------------
class Database:
    """A device-resident database: key-value (one field-major table) or
    order-entry (24 int64 column tables)."""

    def __init__(self, schema: str = "kv", *, n_records: int = 0, n_fields: int = 0,
                 field_bytes: int = 8, n_warehouses: int = 0, order_cap: int = 0,
                 max_ops_per_txn: int = 16, max_batch_txns: int = 1 << 16,
                 max_batch_ops: Optional[int] = None, device: int = 0):
        d = DbDesc()
        d.schema = SCHEMA_KV if schema == "kv" else SCHEMA_ORDER_ENTRY
        d.field_bytes = field_bytes
        d.n_records = n_records
        d.n_fields = n_fields
        d.n_warehouses = n_warehouses
        d.order_cap = order_cap
        d.max_ops_per_txn = max_ops_per_txn
        d.max_batch_txns = max_batch_txns
        d.max_batch_ops = max_batch_ops or max_batch_txns * max_ops_per_txn
        d.device = device
        self.desc = d
        self.schema = schema
        self.handle = gcc_db_create(d)

    def close(self):
        if self.handle:
            gcc_db_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def table_bytes(self, table_id: int = 0) -> int:
        return int(load().gcc_table_bytes(self.handle, table_id))

    def load_table(self, table_id: int, src):
        """Copy a numpy array or a CUDA tensor into a table (resets control words)."""
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src)
            gcc_load_table(self.handle, table_id, _host_ptr(src), src.nbytes, False)
        else:
            gcc_load_table(self.handle, table_id, _tensor_ptr(src),
                           src.numel() * src.element_size(), True)

    def read_table(self, table_id: int = 0, dtype=np.uint64) -> np.ndarray:
        nbytes = self.table_bytes(table_id)
        out = np.empty(nbytes // np.dtype(dtype).itemsize, dtype=dtype)
        gcc_db_read_table(self.handle, table_id, _host_ptr(out), nbytes, False)
        return out

    # key-value helpers -----------------------------------------------------
    def load_kv(self, table: np.ndarray):
        self.load_table(0, table)

    def init_seeded(self, seed: int):
        """Fill the key-value table on the device (see workload.kv_table_seeded)."""
        gcc_init_table_seeded(self.handle, 0, seed)

    def read_kv(self) -> np.ndarray:
        d = self.desc
        t = self.read_table(0)
        return t.reshape(d.n_fields, d.n_records) if d.field_bytes == 8 else \
            t.reshape(d.n_fields, d.n_records, 2)

    # order-entry helpers ---------------------------------------------------
    def load_oe(self, db: dict):
        for i, c in enumerate(wl.OE_COLUMNS):
            self.load_table(i, np.ascontiguousarray(db[c], dtype=np.int64))

    def read_oe(self) -> dict:
        return {c: self.read_table(i, dtype=np.int64) for i, c in enumerate(wl.OE_COLUMNS)}

    # execution -------------------------------------------------------------
    def submit(self, scheme, batch: "wl.KVBatch", p: Optional[ExecParams] = None,
               stream: int = 0) -> "Batch":
        """Host-input submission: inputs are copied before this returns."""
        txns = np.ascontiguousarray(batch.txns)
        ops = np.ascontiguousarray(batch.ops)
        operands = np.ascontiguousarray(batch.operands, dtype=np.uint64)
        h = gcc_txn_batch_submit(self.handle, scheme, _host_ptr(txns), batch.n_txns,
                                 _host_ptr(ops), _host_ptr(operands), batch.n_ops, False, p,
                                 stream)
        return Batch(h, batch.n_txns, batch.n_ops)

    def run(self, scheme, batch, p: Optional[ExecParams] = None, timeout_s: float = 120.0):
        """Submit, wait, and return (results, reads uint64[n_ops, 2], stats)."""
        b = self.submit(scheme, batch, p)
        try:
            return b.wait(timeout_s)
        finally:
            b.free()

    def execute(self, scheme, d_txns, d_ops, d_operands, n_txns: int, n_ops: int, d_results,
                d_reads, p: Optional[ExecParams] = None, stream: int = 0):
        """Device-resident execution on torch CUDA tensors (asynchronous)."""
        gcc_execute(self.handle, scheme, _tensor_ptr(d_txns), n_txns, _tensor_ptr(d_ops),
                    _tensor_ptr(d_operands), n_ops, p, _tensor_ptr(d_results),
                    _tensor_ptr(d_reads), stream)

    def last_stats(self) -> dict:
        return gcc_last_stats(self.handle)

    def stage_history(self, n: int = 256) -> list:
        return gcc_stage_history(self.handle, n)


class Batch:
    def __init__(self, handle: int, n_txns: int, n_ops: int):
        self.handle, self.n_txns, self.n_ops = handle, n_txns, n_ops

    def wait(self, timeout_s: Optional[float] = None, results: Optional[np.ndarray] = None,
             reads: Optional[np.ndarray] = None):
        results = np.zeros(self.n_txns, dtype=wl.RESULT_DTYPE) if results is None else results
        reads = np.zeros((self.n_ops, 2), dtype=np.uint64) if reads is None else reads
        t = WAIT_FOREVER if timeout_s is None else int(timeout_s * 1e9)
        stats = gcc_batch_wait(self.handle, t, _host_ptr(results) if self.n_txns else None,
                               _host_ptr(reads) if self.n_ops else None)
        return results, reads, stats

    def free(self):
        if self.handle:
            gcc_batch_free(self.handle)
            self.handle = 0


class MultiPlan:
    """One persistent launch over several (database, device batch) pairs.

    ``entries`` are (Database, d_txns, n_txns, d_ops, d_operands, n_ops,
    d_results, d_reads) with torch CUDA tensors; the tensors must outlive the
    plan."""

    def __init__(self, scheme, entries, p: Optional[ExecParams] = None):
        self._keep = entries
        bs = [MultiBatch(db.handle, _tensor_ptr(tx), n_t, 0, _tensor_ptr(op), _tensor_ptr(od), n_o,
                         _tensor_ptr(rs), _tensor_ptr(rd))
              for (db, tx, n_t, op, od, n_o, rs, rd) in entries]
        self.n = len(bs)
        self.handle = gcc_multi_plan_create(scheme, bs, p)

    def launch(self, use_graph: bool = True, stream: int = 0):
        gcc_multi_launch(self.handle, use_graph, stream)

    def stats(self, i: int) -> dict:
        return gcc_multi_stats(self.handle, i)

    def close(self):
        if self.handle:
            gcc_multi_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over one or more databases (lanes).

    ``lanes`` are (Database, scheme, max_batch_txns, write_budget_bytes,
    max_delay_ns, depth) tuples; zero budget/delay/depth take the defaults."""

    def __init__(self, lanes, p: Optional[ExecParams] = None):
        arr = (ServerLane * len(lanes))()
        for i, (db, scheme, cap, budget, delay, depth) in enumerate(lanes):
            arr[i] = ServerLane(db.handle, _scheme(scheme), cap, budget, delay, depth, 0)
        self._dbs = [l[0] for l in lanes]
        h = P()
        _check(load().gcc_server_create(arr, len(lanes), ctypes.byref(p) if p is not None else None,
                                        ctypes.byref(h)))
        self.handle = h.value

    @staticmethod
    def now_ns() -> int:
        return int(load().gcc_server_now_ns())

    def enqueue(self, lane: int, txn: np.ndarray, ops: np.ndarray, operands: np.ndarray,
                arrival_ns: int) -> int:
        rid = ctypes.c_uint64(0)
        _check(load().gcc_server_enqueue(self.handle, lane, _host_ptr(txn), _host_ptr(ops),
                                         _host_ptr(operands), arrival_ns, ctypes.byref(rid)))
        return rid.value

    def pump(self):
        _check(load().gcc_server_pump(self.handle))

    def drain(self):
        _check(load().gcc_server_drain(self.handle))

    def completions(self, max_n: int = 1 << 16, reads_capacity: int = 1 << 20):
        out = np.zeros(max_n, dtype=COMPLETION_DTYPE)
        reads = np.zeros((reads_capacity, 2), dtype=np.uint64)
        n = ctypes.c_uint32(0)
        _check(load().gcc_server_completions(self.handle, _host_ptr(out), _host_ptr(reads),
                                             reads_capacity, max_n, ctypes.byref(n)))
        return out[: n.value], reads

    def run_trace(self, lane_of: np.ndarray, batch: "wl.KVBatch", arrival_offset_ns: np.ndarray):
        """Open-loop replay of a trace; returns (completions, reads[n_ops, 2])."""
        n = batch.n_txns
        out = np.zeros(n, dtype=COMPLETION_DTYPE)
        reads = np.zeros((batch.n_ops, 2), dtype=np.uint64)
        lane_of = np.ascontiguousarray(lane_of, dtype=np.uint32)
        arr = np.ascontiguousarray(arrival_offset_ns, dtype=np.uint64)
        _check(load().gcc_server_run_trace(self.handle, n, _host_ptr(lane_of),
                                           _host_ptr(np.ascontiguousarray(batch.txns)),
                                           _host_ptr(np.ascontiguousarray(batch.ops)),
                                           _host_ptr(np.ascontiguousarray(batch.operands)),
                                           _host_ptr(arr), _host_ptr(out), _host_ptr(reads)))
        return out, reads

    def lane_totals(self, lane: int) -> dict:
        c, a, b = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(load().gcc_server_lane_totals(self.handle, lane, ctypes.byref(c), ctypes.byref(a),
                                             ctypes.byref(b)))
        return {"committed": c.value, "aborts": a.value, "batches": b.value}

    def close(self):
        if self.handle:
            _check(load().gcc_server_destroy(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
