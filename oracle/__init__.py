"""CPU oracle for batched OLTP concurrency control -- test infrastructure only.

A plain single-threaded serial executor written in C (``oracle.c``), loaded
through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the engine never does.

Every function follows the serializability contract the paper states for all
of its schemes (Sec. II, Sec. III-E): a batch's outcome must equal the serial
execution of its committed transactions in some order, which the engine
reports as a commit order.  ``replay_check`` checks exactly that; ``serial``
executes an order directly (transaction-id order is the deterministic
scheme's, Sec. II-C); ``brute_force`` enumerates every serial order of a tiny
batch.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c")]
_lock = threading.Lock()
_lib = None

ST_PENDING, ST_COMMITTED, ST_TIMEOUT, ST_INVALID = 0, 1, 2, 3
ERRORS = {0: "ok", 1: "bad key", 2: "bad field", 3: "bad kind", 4: "bad commit order",
          5: "too many txns", 6: "out of memory", 7: "bad txn type",
          8: "not all committed", 9: "bad insert"}


def build(out: str = _SO, cflags=None) -> str:
    """Compile the oracle with gcc into ``out`` (plain C11, portable flags)."""
    flags = cflags or ["-O2"]
    cmd = ["gcc", "-std=c11", *flags, "-fPIC", "-shared", "-o", out, *_SRC]
    subprocess.run(cmd, check=True, cwd=_HERE)
    return out


def _stale() -> bool:
    if not os.path.exists(_SO):
        return True
    t = os.path.getmtime(_SO)
    return any(os.path.getmtime(p) > t for p in _SRC + [os.path.join(_HERE, "oracle.h")])


class Report(ctypes.Structure):
    _fields_ = [("err", ctypes.c_int32), ("n_committed", ctypes.c_uint32),
                ("n_read_mismatch", ctypes.c_uint64), ("first_bad_op", ctypes.c_uint64),
                ("n_table_mismatch", ctypes.c_uint64), ("first_bad_word", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KV(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("nrec", ctypes.c_uint64),
                ("nfields", ctypes.c_uint32), ("field_bytes", ctypes.c_uint32)]


OE_COLUMNS = ["w_ytd", "w_tax", "d_ytd", "d_tax", "d_next_o_id", "c_balance",
              "c_ytd_payment", "c_payment_cnt", "c_discount", "i_price", "s_quantity",
              "s_ytd", "s_order_cnt", "s_remote_cnt", "o_c_id", "o_ol_cnt", "o_all_local",
              "no_flag", "ol_i_id", "ol_supply_w_id", "ol_quantity", "ol_amount",
              "c_last", "c_first"]


class OE(ctypes.Structure):
    _fields_ = [("W", ctypes.c_uint32), ("order_cap", ctypes.c_uint32)] + \
               [(c, ctypes.c_void_p) for c in OE_COLUMNS]


def load(path: str | None = None):
    """Load (building first if missing or stale) the oracle library."""
    global _lib
    with _lock:
        if path is not None:
            return _bind(ctypes.CDLL(path))
        if _lib is None:
            if _stale():
                build()
            _lib = _bind(ctypes.CDLL(_SO))
        return _lib


def _bind(lib):
    P = ctypes.c_void_p
    lib.orc_kv_serial.argtypes = [ctypes.POINTER(KV), P, ctypes.c_uint32, P, P, P,
                                  ctypes.c_uint32, P]
    lib.orc_kv_serial.restype = ctypes.c_int
    lib.orc_commit_sequence.argtypes = [P, ctypes.c_uint32, P, ctypes.POINTER(ctypes.c_uint32)]
    lib.orc_commit_sequence.restype = ctypes.c_int
    lib.orc_kv_replay_check.argtypes = [ctypes.POINTER(KV), P, P, ctypes.c_uint32, P, P, P, P,
                                        ctypes.c_int, ctypes.POINTER(Report)]
    lib.orc_kv_replay_check.restype = ctypes.c_int
    lib.orc_kv_brute_force.argtypes = [ctypes.POINTER(KV), P, ctypes.c_uint32, P, P, P, P, P]
    lib.orc_kv_brute_force.restype = ctypes.c_int64
    lib.orc_kv_sum.argtypes = [ctypes.POINTER(KV), P]
    lib.orc_kv_sum.restype = None
    lib.orc_oe_serial.argtypes = [ctypes.POINTER(OE), P, ctypes.c_uint32, P, P, P,
                                  ctypes.c_uint32, P]
    lib.orc_oe_serial.restype = ctypes.c_int
    lib.orc_oe_check_consistency.argtypes = [ctypes.POINTER(OE)]
    lib.orc_oe_check_consistency.restype = ctypes.c_int
    return lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _kv(table: np.ndarray, field_bytes: int) -> KV:
    nfields, nrec = table.shape[0], table.shape[1]
    return KV(table.ctypes.data, nrec, nfields, field_bytes)


def _field_bytes(table: np.ndarray) -> int:
    return 16 if table.ndim == 3 else 8


def _check(e: int, what: str):
    if e != 0:
        raise OracleError(f"{what}: {ERRORS.get(e, e)}")


class OracleError(RuntimeError):
    pass


def serial(table: np.ndarray, batch, order=None, lib=None):
    """Execute ``batch`` serially on a copy of ``table`` in ``order`` (default:
    transaction-id order).  Returns (final table, reads uint64[n_ops, 2])."""
    lib = lib or load()
    work = np.ascontiguousarray(table).copy()
    reads = np.zeros((batch.n_ops, 2), dtype=np.uint64)
    kv = _kv(work, _field_bytes(work))
    o = None if order is None else np.ascontiguousarray(order, dtype=np.uint32)
    e = lib.orc_kv_serial(ctypes.byref(kv), _p(batch.txns), batch.n_txns, _p(batch.ops),
                          _p(batch.operands), _p(o), 0 if o is None else o.size, _p(reads))
    _check(e, "serial execution")
    return work, reads


def serial_inplace(table: np.ndarray, batch, order=None, lib=None):
    """Serial execution directly on ``table`` without recording reads (the
    benchmark's CPU baseline times this call)."""
    lib = lib or load()
    kv = _kv(table, _field_bytes(table))
    o = None if order is None else np.ascontiguousarray(order, dtype=np.uint32)
    e = lib.orc_kv_serial(ctypes.byref(kv), _p(batch.txns), batch.n_txns, _p(batch.ops),
                          _p(batch.operands), _p(o), 0 if o is None else o.size, None)
    _check(e, "serial execution")


def commit_sequence(results: np.ndarray, lib=None) -> np.ndarray:
    """Committed transaction ids in reported commit order (checks permutation)."""
    lib = lib or load()
    order = np.zeros(max(1, results.size), dtype=np.uint32)
    nc = ctypes.c_uint32(0)
    e = lib.orc_commit_sequence(_p(results), results.size, _p(order), ctypes.byref(nc))
    _check(e, "commit sequence")
    return order[: nc.value].copy()


def replay_check(init_table: np.ndarray, gpu_table: np.ndarray, batch, results: np.ndarray,
                 gpu_reads: np.ndarray, require_all: bool = True, lib=None,
                 inplace: bool = False) -> dict:
    """Replay committed txns in commit order from ``init_table`` and compare.

    Returns the report dict; ``ok`` is True when every read value and every
    word of the final table match bit for bit."""
    lib = lib or load()
    work = init_table if inplace else np.ascontiguousarray(init_table).copy()
    kv = _kv(work, _field_bytes(work))
    rep = Report()
    lib.orc_kv_replay_check(ctypes.byref(kv), _p(np.ascontiguousarray(gpu_table)),
                            _p(batch.txns), batch.n_txns, _p(batch.ops), _p(batch.operands),
                            _p(np.ascontiguousarray(results)),
                            _p(np.ascontiguousarray(gpu_reads)), int(require_all),
                            ctypes.byref(rep))
    d = rep.as_dict()
    d["error"] = ERRORS.get(d["err"], d["err"])
    d["ok"] = (d["err"] == 0 and d["n_read_mismatch"] == 0 and d["n_table_mismatch"] == 0)
    return d


def brute_force(init_table: np.ndarray, batch, obs_table: np.ndarray, obs_reads: np.ndarray,
                lib=None):
    """(number of serial orders reproducing the observation, first such order)."""
    lib = lib or load()
    kv = _kv(np.ascontiguousarray(init_table), _field_bytes(init_table))
    first = np.zeros(8, dtype=np.uint32)
    n = lib.orc_kv_brute_force(ctypes.byref(kv), _p(batch.txns), batch.n_txns, _p(batch.ops),
                               _p(batch.operands), _p(np.ascontiguousarray(obs_reads)),
                               _p(np.ascontiguousarray(obs_table)), _p(first))
    if n < 0:
        raise OracleError(f"brute force: {ERRORS.get(-n, -n)}")
    return int(n), first[: batch.n_txns].copy()


def table_sum(table: np.ndarray, lib=None):
    """(lane-0 sum mod 2^64, lane-1 u16 sum mod 2^16) of a key-value table."""
    lib = lib or load()
    kv = _kv(np.ascontiguousarray(table), _field_bytes(table))
    out = np.zeros(2, dtype=np.uint64)
    lib.orc_kv_sum(ctypes.byref(kv), _p(out))
    return int(out[0]), int(out[1])


# ---------------------------------------------------------------------------
# order-entry
# ---------------------------------------------------------------------------
def _oe(db: dict, W: int, order_cap: int) -> OE:
    s = OE(W, order_cap)
    for c in OE_COLUMNS:
        a = db[c]
        assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
        setattr(s, c, a.ctypes.data)
    return s


def oe_serial(db: dict, W: int, order_cap: int, batch, order=None, lib=None):
    """Serial execution of an order-entry batch on a copy of ``db`` (a dict of
    int64 column arrays).  Returns (final db, reads uint64[n_ops, 2])."""
    lib = lib or load()
    work = {c: np.ascontiguousarray(db[c]).copy() for c in OE_COLUMNS}
    s = _oe(work, W, order_cap)
    reads = np.zeros((batch.n_ops, 2), dtype=np.uint64)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.uint32)
    e = lib.orc_oe_serial(ctypes.byref(s), _p(batch.txns), batch.n_txns, _p(batch.ops),
                          _p(batch.operands), _p(o), 0 if o is None else o.size, _p(reads))
    _check(e, "order-entry serial execution")
    return work, reads


def oe_consistency(db: dict, W: int, order_cap: int, lib=None) -> int:
    """Bit mask of violated order-entry consistency conditions (0 = consistent)."""
    lib = lib or load()
    return int(lib.orc_oe_check_consistency(ctypes.byref(_oe(db, W, order_cap))))


def oe_replay_check(init_db: dict, gpu_db: dict, W: int, order_cap: int, batch,
                    results: np.ndarray, gpu_reads: np.ndarray, lib=None) -> dict:
    """Replay committed order-entry txns in commit order and compare every read
    of a committed txn and every column of the final database."""
    order = commit_sequence(results, lib=lib)
    final, reads = oe_serial(init_db, W, order_cap, batch, order=order, lib=lib)
    committed = results["status"] == ST_COMMITTED
    op_mask = np.repeat(committed, batch.txns["n_ops"].astype(np.int64))
    bad_reads = int(np.count_nonzero(np.any(reads[op_mask] != gpu_reads[op_mask], axis=1)))
    bad_cols = {c: int(np.count_nonzero(final[c] != gpu_db[c])) for c in OE_COLUMNS}
    bad_cols = {c: n for c, n in bad_cols.items() if n}
    return {"ok": bad_reads == 0 and not bad_cols, "n_committed": int(order.size),
            "n_read_mismatch": bad_reads, "bad_columns": bad_cols}


def customer_by_last_name(c_last, c_first, name: int) -> int:
    """The customer a payment by last name selects in one district, given the
    district's last-name ids and first-name keys: among the customers named
    ``name``, ordered by first name and then by customer index, the one at
    position ceil(n/2) (1-based) -- the middle one, the lower of the two
    middles for an even n.  Returns its index in the district, or -1 when
    nobody has the name.  (The by-name variant of the order-entry payment;
    its selection rule is this library's reading, the paper's Sec. IV-A
    naming only the transaction.)"""
    named = [c for c in range(len(c_last)) if int(c_last[c]) == name]
    if not named:
        return -1
    named.sort(key=lambda c: (int(c_first[c]), c))
    return named[(len(named) + 1) // 2 - 1]

