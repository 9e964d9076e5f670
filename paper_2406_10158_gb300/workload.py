"""Seeded synthetic inputs for the transaction engine and its oracle.

This module only *defines inputs*: initial table contents and transaction
batches.  It contains none of the concurrency-control arithmetic and none of
the operation semantics (what a READ or a read-modify-write does to a record);
those live separately in the CUDA engine and in the CPU oracle, which share no
code.  Both sides consume the arrays built here.

Workload shapes follow the paper's experimental setup (Sec. IV-A): YCSB-style
key-value transactions of 16 single-record accesses over a Zipfian key
distribution with a write fraction W and contention parameter theta, and a
TPC-C-style order-entry mix of NewOrder and Payment (generated by
``order_entry``).  The benchmark suites themselves are not used: everything is
regenerated from seeds.

Array formats (little-endian, matching ``include/gcc_gb300.h``):

* ``TXN_DTYPE``  -- one 8-byte record per transaction: first_op (u32), n_ops
  (u16), type (u16).  Transactions are listed in transaction-id order and their
  op ranges are increasing in id order.
* ``OP_DTYPE``   -- one 8-byte descriptor per op: key (u32), field (u8),
  kind (u8), aux (u16).
* operands      -- ``uint64[n_ops, 2]``: (lo, hi) per op.
* KV tables     -- field-major ("columnar"): ``uint64[nfields, nrec]`` for
  8-byte fields, ``uint64[nfields, nrec, 2]`` for 16-byte slots (bytes 0-7 in
  lo, bytes 8-15 in hi; only bytes 0-9 carry payload).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# ---------------------------------------------------------------------------
# record formats shared with the C ABI
# ---------------------------------------------------------------------------
TXN_DTYPE = np.dtype([("first_op", "<u4"), ("n_ops", "<u2"), ("type", "<u2")])
OP_DTYPE = np.dtype([("key", "<u4"), ("field", "u1"), ("kind", "u1"), ("aux", "<u2")])
RESULT_DTYPE = np.dtype([("status", "<u4"), ("attempts", "<u4"), ("commit_order", "<u8")])

# op kinds (values fixed by the C ABI)
OP_READ = 0
OP_ADD = 1

# transaction types
TXN_KV = 0
TXN_NEW_ORDER = 1
TXN_PAYMENT = 2

MASK64 = (1 << 64) - 1

# ---------------------------------------------------------------------------
# splitmix64 (Steele, Lea, Flood: "Fast splittable pseudorandom number
# generators", OOPSLA 2014; constants as published there and in Vigna's
# reference C code).  Used for the closed-form initial values of the small
# key-value store and for deriving stream seeds.
# ---------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64_at(seed: int, counter) -> np.ndarray:
    """The ``counter``-th output (1-based) of splitmix64 seeded with ``seed``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + _GOLDEN * c
    return _mix64(z)


def splitmix64_init(seed: int, key, field, nfields: int) -> np.ndarray:
    """Initial value of (key, field): splitmix64 output number key*nfields+field+1."""
    k = np.asarray(key, dtype=np.uint64)
    f = np.asarray(field, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = k * np.uint64(nfields) + f + np.uint64(1)
    return splitmix64_at(seed, ctr)


def derive_seed(seed: int, stream: int) -> int:
    return int(splitmix64_at(seed, np.uint64(stream + 1)))


# ---------------------------------------------------------------------------
# key distributions
# ---------------------------------------------------------------------------
_ZETA_CACHE: dict = {}


def _zeta(n: int, theta: float) -> float:
    key = (n, theta)
    if key not in _ZETA_CACHE:
        total = 0.0
        step = 1 << 22
        for lo in range(1, n + 1, step):
            i = np.arange(lo, min(n, lo + step - 1) + 1, dtype=np.float64)
            total += float(np.sum(i ** (-theta)))
        _ZETA_CACHE[key] = total
    return _ZETA_CACHE[key]


def zipf_ranks(rng: np.random.Generator, n_items: int, theta: float, size) -> np.ndarray:
    """Zipfian ranks in [0, n_items) by the closed-form inversion of Gray et al.,
    "Quickly generating billion-record synthetic databases" (SIGMOD 1994), the
    generator YCSB uses.  theta = 0 gives the uniform distribution; rank 0 is
    the hottest item."""
    size = tuple(np.atleast_1d(size))
    if theta == 0.0:
        return rng.integers(0, n_items, size=size, dtype=np.int64).astype(np.uint64)
    zetan = _zeta(n_items, theta)
    zeta2 = 1.0 + 2.0 ** (-theta)
    alpha = 1.0 / (1.0 - theta)
    eta = (1.0 - (2.0 / n_items) ** (1.0 - theta)) / (1.0 - zeta2 / zetan)
    u = rng.random(size=size)
    uz = u * zetan
    r = np.floor(n_items * np.power(eta * u - eta + 1.0, alpha))
    r = np.clip(r, 0, n_items - 1)
    r = np.where(uz < 1.0 + 0.5 ** theta, 1.0, r)
    r = np.where(uz < 1.0, 0.0, r)
    return r.astype(np.uint64)


def feistel_permute(x: np.ndarray, n_items: int, seed: int) -> np.ndarray:
    """A seeded bijection of [0, n_items): a 4-round balanced Feistel network on
    the smallest even bit width covering n_items, with cycle walking for values
    that land outside the range.  It scatters Zipf ranks over the key space so
    that hot keys are not adjacent."""
    bits = max(2, int(math.ceil(math.log2(max(n_items, 2)))))
    if bits % 2:
        bits += 1
    half = bits // 2
    hmask = np.uint64((1 << half) - 1)
    rkeys = [np.uint64(derive_seed(seed, 100 + r)) for r in range(4)]

    def one_pass(v):
        lo = v & hmask
        hi = v >> np.uint64(half)
        for rk in rkeys:
            with np.errstate(over="ignore"):
                f = _mix64(lo ^ rk) & hmask
            lo, hi = hi ^ f, lo
        return (hi << np.uint64(half)) | lo

    v = np.asarray(x, dtype=np.uint64)
    out = one_pass(v)
    bad = out >= np.uint64(n_items)
    while np.any(bad):
        out[bad] = one_pass(out[bad])
        bad = out >= np.uint64(n_items)
    return out


def distinct_rows(draw, n_rows: int, width: int) -> np.ndarray:
    """An (n_rows, width) array from ``draw(shape)`` with distinct values per
    row: duplicates (after the first occurrence) are redrawn until none remain."""
    a = draw((n_rows, width))
    while True:
        order = np.argsort(a, axis=1, kind="stable")
        s = np.take_along_axis(a, order, axis=1)
        dup_sorted = np.zeros_like(s, dtype=bool)
        dup_sorted[:, 1:] = s[:, 1:] == s[:, :-1]
        if not dup_sorted.any():
            return a
        dup = np.zeros_like(dup_sorted)
        np.put_along_axis(dup, order, dup_sorted, axis=1)
        rows, cols = np.nonzero(dup)
        a[rows, cols] = draw((rows.size,))


# ---------------------------------------------------------------------------
# key-value workloads
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class KVBatch:
    """A batch of key-value transactions (see module docstring for formats)."""
    txns: np.ndarray        # TXN_DTYPE[n_txns]
    ops: np.ndarray         # OP_DTYPE[n_ops]
    operands: np.ndarray    # uint64[n_ops, 2]

    @property
    def n_txns(self) -> int:
        return int(self.txns.shape[0])

    @property
    def n_ops(self) -> int:
        return int(self.ops.shape[0])


def kv_table_splitmix(seed: int, nrec: int, nfields: int) -> np.ndarray:
    """uint64[nfields, nrec] with value(key, field) = splitmix64_init(seed, key, field)."""
    keys = np.arange(nrec, dtype=np.uint64)
    out = np.empty((nfields, nrec), dtype=np.uint64)
    for f in range(nfields):
        out[f] = splitmix64_init(seed, keys, f, nfields)
    return out


def kv_table_seeded(seed: int, nrec: int, nfields: int, field_bytes: int = 8) -> np.ndarray:
    """The table gcc_init_table_seeded writes on the device: 8-byte slots as
    kv_table_splitmix; 16-byte slots (uint64[nfields, nrec, 2]) hold that value
    in bytes 0-7 and the low 16 bits of the same output number under the seed
    splitmix64(seed, 2) in bytes 8-9."""
    lo = kv_table_splitmix(seed, nrec, nfields)
    if field_bytes == 8:
        return lo
    hi = kv_table_splitmix(int(splitmix64_at(seed, 2)), nrec, nfields) & np.uint64(0xFFFF)
    return np.stack([lo, hi], axis=-1)


def kv_table_bytes(seed: int, nrec: int, nfields: int, payload_bytes: int = 10) -> np.ndarray:
    """uint64[nfields, nrec, 2]: 16-byte slots whose first ``payload_bytes``
    bytes are uniform random and whose remaining bytes are zero."""
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 7)))
    out = np.zeros((nfields, nrec, 2), dtype=np.uint64)
    raw = out.view(np.uint8).reshape(nfields, nrec, 16)
    for f in range(nfields):
        raw[f, :, :payload_bytes] = np.frombuffer(
            rng.bytes(nrec * payload_bytes), dtype=np.uint8).reshape(nrec, payload_bytes)
    return out


def kv_batch(seed: int, *, nrec: int, nfields: int, n_txns: int, ops_per_txn=16,
             read_ratio: float = 0.5, theta: float = 0.0, field_bytes: int = 8,
             delta_range=(-1000, 1000), permute_keys: Optional[bool] = None,
             ops_range: Optional[tuple] = None) -> KVBatch:
    """A batch of YCSB-style transactions.

    Each transaction accesses ``ops_per_txn`` distinct keys (or a per-txn count
    uniform in ``ops_range`` inclusive).  Keys are Zipfian(theta) ranks passed
    through a seeded Feistel permutation (theta = 0: uniform).  Each op is a
    READ with probability ``read_ratio``, else an ADD; its field is uniform.
    8-byte fields get an int64 delta uniform in ``delta_range`` (two's
    complement); 16-byte slots get a (u64, u16) delta uniform over both lanes.
    """
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 1)))
    if ops_range is not None:
        counts = rng.integers(ops_range[0], ops_range[1] + 1, size=n_txns).astype(np.int64)
    else:
        counts = np.full(n_txns, ops_per_txn, dtype=np.int64)
    width = int(counts.max()) if n_txns else 0
    if width > nrec:
        raise ValueError("more ops per transaction than records")
    if permute_keys is None:
        permute_keys = theta > 0.0
    perm_seed = derive_seed(seed, 2)

    def draw(shape):
        r = zipf_ranks(rng, nrec, theta, shape)
        return feistel_permute(r, nrec, perm_seed) if permute_keys else r

    keys2d = distinct_rows(draw, n_txns, width) if n_txns else np.zeros((0, 0), np.uint64)
    valid = np.arange(width)[None, :] < counts[:, None]
    n_ops = int(counts.sum())
    txns = np.zeros(n_txns, dtype=TXN_DTYPE)
    first = np.zeros(n_txns, dtype=np.int64)
    if n_txns:
        first[1:] = np.cumsum(counts)[:-1]
    txns["first_op"] = first.astype(np.uint32)
    txns["n_ops"] = counts.astype(np.uint16)
    txns["type"] = TXN_KV
    ops = np.zeros(n_ops, dtype=OP_DTYPE)
    ops["key"] = keys2d[valid].astype(np.uint32)
    ops["field"] = rng.integers(0, nfields, size=n_ops).astype(np.uint8)
    is_read = rng.random(n_ops) < read_ratio
    ops["kind"] = np.where(is_read, OP_READ, OP_ADD).astype(np.uint8)
    operands = np.zeros((n_ops, 2), dtype=np.uint64)
    if field_bytes == 8:
        d = rng.integers(delta_range[0], delta_range[1] + 1, size=n_ops, dtype=np.int64)
        operands[:, 0] = d.view(np.uint64)
    else:
        operands[:, 0] = rng.integers(0, 1 << 64, size=n_ops, dtype=np.uint64)
        operands[:, 1] = rng.integers(0, 1 << 16, size=n_ops, dtype=np.uint64)
    operands[is_read] = 0
    return KVBatch(txns=txns, ops=ops, operands=operands)


def kv_batch_from_lists(txn_ops, field_bytes: int = 8) -> KVBatch:
    """A batch from explicit per-transaction lists of (key, field, kind, lo, hi)."""
    n_ops = sum(len(t) for t in txn_ops)
    txns = np.zeros(len(txn_ops), dtype=TXN_DTYPE)
    ops = np.zeros(n_ops, dtype=OP_DTYPE)
    operands = np.zeros((n_ops, 2), dtype=np.uint64)
    i = 0
    for t, lst in enumerate(txn_ops):
        txns[t] = (i, len(lst), TXN_KV)
        for (key, field, kind, lo, hi) in lst:
            ops[i] = (key, field, kind, 0)
            operands[i, 0] = lo & MASK64
            operands[i, 1] = hi & MASK64
            i += 1
    return KVBatch(txns=txns, ops=ops, operands=operands)


# ---------------------------------------------------------------------------
# named key-value configurations (the paper's YCSB shapes, Sec. IV-A)
# ---------------------------------------------------------------------------
SEEDS = (0x5EED0001, 0x5EED0002, 0x5EED0003, 0x5EED0004, 0x5EED0005)


def small_kv(seed: int = SEEDS[0], n_txns: int = 4096, nrec: int = 65536):
    """65,536 records x 8 u64 fields (splitmix64 init), 4,096 txns x 16 distinct
    uniform keys, 50% reads / 50% ADD of an int64 delta in [-1000, 1000]."""
    table = kv_table_splitmix(seed, nrec, 8)
    batch = kv_batch(derive_seed(seed, 11), nrec=nrec, nfields=8, n_txns=n_txns,
                     ops_per_txn=16, read_ratio=0.5, theta=0.0, field_bytes=8)
    return table, batch


def ycsb_kv(seed: int = SEEDS[1], *, theta: float = 0.8, read_ratio: float = 0.5,
            nrec: int = 1 << 24, n_txns: int = 1 << 20, nfields: int = 10,
            with_table: bool = True):
    """2^24 records x 10 fields of 10 payload bytes in 16-byte slots; 2^20 txns
    x 16 distinct Zipfian keys over a seeded permutation."""
    table = kv_table_bytes(seed, nrec, nfields) if with_table else None
    batch = kv_batch(derive_seed(seed, int(theta * 1000) * 10 + int(read_ratio * 100)),
                     nrec=nrec, nfields=nfields, n_txns=n_txns, ops_per_txn=16,
                     read_ratio=read_ratio, theta=theta, field_bytes=16)
    return table, batch


def kv_hotspot(seed: int = SEEDS[1], *, hot_frac: float = 0.1, nrec: int = 1 << 24,
               n_txns: int = 1 << 20, nfields: int = 10, hot_key: int = 12345,
               with_table: bool = True):
    """The key-value shape of ``ycsb_kv`` with uniform keys (read ratio 0.5),
    except that a ``hot_frac`` share of the transactions (drawn with their
    own seed) turn their first op into an ADD on record ``hot_key``: one hot
    spot among cold records.  Transactions that already touch ``hot_key``
    are left as they are, so keys stay distinct within a transaction."""
    table = kv_table_bytes(seed, nrec, nfields) if with_table else None
    batch = kv_batch(derive_seed(seed, 7001), nrec=nrec, nfields=nfields, n_txns=n_txns,
                     ops_per_txn=16, read_ratio=0.5, theta=0.0, field_bytes=16)
    rng = np.random.default_rng(derive_seed(seed, 7002))
    pick = np.nonzero(rng.random(n_txns) < hot_frac)[0]
    keys = batch.ops["key"].reshape(n_txns, 16)
    pick = pick[~(keys[pick] == hot_key).any(axis=1)]
    first = batch.txns["first_op"][pick].astype(np.int64)
    batch.ops["key"][first] = hot_key
    batch.ops["kind"][first] = OP_ADD
    return table, batch


# ---------------------------------------------------------------------------
# order-entry workloads (TPC-C-shaped NewOrder / Payment, Sec. IV-A)
# ---------------------------------------------------------------------------
# op kinds (values fixed by the C ABI)
OE_W_READ, OE_W_PAY, OE_D_NEWORDER, OE_D_PAY = 16, 17, 18, 19
OE_C_READ, OE_C_PAY, OE_I_READ, OE_S_NEWORDER = 20, 21, 22, 23
OE_C_PAY_BY_NAME = 24

OE_DISTRICTS = 10
OE_CUSTOMERS = 3000
OE_ITEMS = 100000
OE_MAX_LINES = 15
OE_INITIAL_ORDERS = 3000

OE_COLUMNS = ("w_ytd", "w_tax", "d_ytd", "d_tax", "d_next_o_id", "c_balance",
              "c_ytd_payment", "c_payment_cnt", "c_discount", "i_price", "s_quantity",
              "s_ytd", "s_order_cnt", "s_remote_cnt", "o_c_id", "o_ol_cnt", "o_all_local",
              "no_flag", "ol_i_id", "ol_supply_w_id", "ol_quantity", "ol_amount",
              "c_last", "c_first")


def oe_column_rows(W: int, order_cap: int) -> dict:
    """Number of rows of every order-entry column."""
    n_d = W * OE_DISTRICTS
    rows = {"w": W, "d": n_d, "c": n_d * OE_CUSTOMERS, "i": OE_ITEMS, "s": W * OE_ITEMS,
            "o": n_d * order_cap, "n": n_d * order_cap, "l": n_d * order_cap * OE_MAX_LINES}
    table = {"w_": "w", "d_": "d", "c_": "c", "i_": "i", "s_": "s", "o_": "o", "no": "n",
             "ol": "l"}
    return {c: rows[table[c[:2]]] for c in OE_COLUMNS}


def nurand(rng: np.random.Generator, A: int, x: int, y: int, C: int, size) -> np.ndarray:
    """Non-uniform random integers in [x, y]: ((rand[0,A] | rand[x,y]) + C) mod
    (y - x + 1) + x, the skewed id distribution of the TPC-C workload."""
    a = rng.integers(0, A + 1, size=size, dtype=np.int64)
    b = rng.integers(x, y + 1, size=size, dtype=np.int64)
    return ((a | b) + C) % (y - x + 1) + x


OE_LAST_NAMES = 1000


def oe_customer_names(seed: int, W: int) -> dict:
    """Name keys of every customer, rows as the c_ columns: ``c_last`` a
    last-name id in [0, 1000) -- the first 1,000 customers of each district
    take ids 0..999 in order, the rest NURand(255, 0, 999), so that every name
    exists in every district and a few are common -- and ``c_first`` a
    uniform 32-bit first-name key.  (Names are ids: the engine keeps no
    strings.)"""
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 22)))
    n_d = W * OE_DISTRICTS
    c_run = int(rng.integers(0, 256))
    last = np.empty((n_d, OE_CUSTOMERS), dtype=np.int64)
    last[:, :OE_LAST_NAMES] = np.arange(OE_LAST_NAMES)
    last[:, OE_LAST_NAMES:] = nurand(rng, 255, 0, OE_LAST_NAMES - 1, c_run,
                                     (n_d, OE_CUSTOMERS - OE_LAST_NAMES))
    first = rng.integers(0, 1 << 32, size=n_d * OE_CUSTOMERS, dtype=np.int64)
    return {"c_last": last.ravel(), "c_first": first}


def oe_initial_db(seed: int, W: int, order_cap: int) -> dict:
    """The initial order-entry database as a dict of int64 columns.

    Money is int64 cents, taxes and discounts basis points.  Each district
    starts with 3,000 orders (ids 1..3000, the last 900 undelivered, i.e. with
    a new-order flag) and d_next_o_id = 3001; w_ytd equals the sum of its
    districts' d_ytd."""
    if order_cap < OE_INITIAL_ORDERS:
        raise ValueError("order_cap below the initial 3,000 orders per district")
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 21)))
    rows = oe_column_rows(W, order_cap)
    db = {c: np.zeros(rows[c], dtype=np.int64) for c in OE_COLUMNS}
    n_d = W * OE_DISTRICTS
    db["w_tax"][:] = rng.integers(0, 2001, size=W)
    db["d_tax"][:] = rng.integers(0, 2001, size=n_d)
    db["d_ytd"][:] = rng.integers(0, 10_000_001, size=n_d)
    db["w_ytd"][:] = db["d_ytd"].reshape(W, OE_DISTRICTS).sum(axis=1)
    db["d_next_o_id"][:] = OE_INITIAL_ORDERS + 1
    n_c = rows["c_balance"]
    db["c_balance"][:] = rng.integers(-100_000, 100_001, size=n_c)
    db["c_ytd_payment"][:] = rng.integers(0, 1_000_001, size=n_c)
    db["c_payment_cnt"][:] = rng.integers(1, 11, size=n_c)
    db["c_discount"][:] = rng.integers(0, 5001, size=n_c)
    db["i_price"][:] = rng.integers(100, 10_001, size=OE_ITEMS)
    db["s_quantity"][:] = rng.integers(10, 101, size=W * OE_ITEMS)
    names = oe_customer_names(seed, W)               # its own stream
    db["c_last"][:] = names["c_last"]
    db["c_first"][:] = names["c_first"]
    # initial orders
    o = np.arange(OE_INITIAL_ORDERS)
    slots = (np.arange(n_d)[:, None] * order_cap + o[None, :]).ravel()
    cnt = rng.integers(5, 16, size=slots.size)
    db["o_c_id"][slots] = rng.integers(0, OE_CUSTOMERS, size=slots.size)
    db["o_ol_cnt"][slots] = cnt
    db["o_all_local"][slots] = 1
    db["no_flag"][slots] = (np.tile(o, n_d) >= 2100).astype(np.int64)
    lines = np.arange(OE_MAX_LINES)
    present = lines[None, :] < cnt[:, None]
    ol = (slots[:, None] * OE_MAX_LINES + lines[None, :])[present]
    dist_of_slot = np.repeat(np.arange(n_d), OE_INITIAL_ORDERS)
    w_of_line = np.repeat(dist_of_slot // OE_DISTRICTS, cnt)
    db["ol_i_id"][ol] = rng.integers(0, OE_ITEMS, size=ol.size)
    db["ol_supply_w_id"][ol] = w_of_line
    db["ol_quantity"][ol] = 5
    delivered = np.repeat(np.tile(o, n_d) < 2100, cnt)
    db["ol_amount"][ol] = np.where(delivered, rng.integers(1, 1_000_000, size=ol.size), 0)
    return db


def oe_batch(seed: int, W: int, n_txns: int, new_order_frac: float = 0.5,
             remote_line_frac: float = 0.01, remote_customer_frac: float = 0.15,
             by_name_frac: float = 0.0) -> KVBatch:
    """A mix of NewOrder and Payment transactions encoded as op lists (layout
    documented with the order-entry op kinds in the C ABI header).

    NewOrder: home warehouse/district uniform, customer NURand(1023), 5-15
    lines with distinct NURand(8191) items, quantity 1-10, each line supplied
    by another warehouse with probability ``remote_line_frac`` when W > 1.
    Payment: amount uniform in [100, 500000] cents; the customer belongs to
    another warehouse with probability ``remote_customer_frac`` when W > 1,
    and is named by last name (op OE_C_PAY_BY_NAME: key = the customer's
    district, aux = a NURand(255, 0, 999) last-name id) with probability
    ``by_name_frac`` (TPC-C's share is 60%), else by id.  The by-name draws
    come after all others, so by_name_frac = 0 gives the same batch as
    before the option existed."""
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 31)))
    c_item = int(rng.integers(0, 8192))
    c_cust = int(rng.integers(0, 1024))
    is_no = rng.random(n_txns) < new_order_frac
    n_no = int(is_no.sum())
    n_pay = n_txns - n_no
    w = rng.integers(0, W, size=n_txns)
    d = rng.integers(0, OE_DISTRICTS, size=n_txns)
    dist = w * OE_DISTRICTS + d
    cust = nurand(rng, 1023, 1, OE_CUSTOMERS, c_cust, n_txns) - 1

    # NewOrder parameters
    ol_cnt = rng.integers(5, OE_MAX_LINES + 1, size=n_no)
    items = distinct_rows(lambda s: nurand(rng, 8191, 1, OE_ITEMS, c_item, s) - 1,
                          n_no, OE_MAX_LINES)
    qty = rng.integers(1, 11, size=(n_no, OE_MAX_LINES))
    w_no = w[is_no]
    supply = np.repeat(w_no[:, None], OE_MAX_LINES, axis=1)
    if W > 1:
        remote = rng.random((n_no, OE_MAX_LINES)) < remote_line_frac
        other = (w_no[:, None] + rng.integers(1, W, size=(n_no, OE_MAX_LINES))) % W
        supply = np.where(remote, other, supply)
    # Payment parameters
    h = rng.integers(100, 500_001, size=n_pay)
    w_pay, d_pay, c_pay = w[~is_no], d[~is_no], cust[~is_no]
    c_w, c_d = w_pay.copy(), d_pay.copy()
    if W > 1:
        rem = rng.random(n_pay) < remote_customer_frac
        c_w = np.where(rem, (w_pay + rng.integers(1, W, size=n_pay)) % W, c_w)
        c_d = np.where(rem, rng.integers(0, OE_DISTRICTS, size=n_pay), c_d)

    n_ops_t = np.where(is_no, 0, 3)
    n_ops_t[is_no] = 3 + 2 * ol_cnt
    first = np.zeros(n_txns, dtype=np.int64)
    if n_txns:
        first[1:] = np.cumsum(n_ops_t)[:-1]
    n_ops = int(n_ops_t.sum())
    txns = np.zeros(n_txns, dtype=TXN_DTYPE)
    txns["first_op"] = first
    txns["n_ops"] = n_ops_t
    txns["type"] = np.where(is_no, TXN_NEW_ORDER, TXN_PAYMENT)
    ops = np.zeros(n_ops, dtype=OP_DTYPE)
    operands = np.zeros((n_ops, 2), dtype=np.uint64)

    # NewOrder head ops
    f_no = first[is_no]
    ops["kind"][f_no] = OE_W_READ
    ops["key"][f_no] = w_no
    ops["kind"][f_no + 1] = OE_D_NEWORDER
    ops["key"][f_no + 1] = dist[is_no]
    ops["kind"][f_no + 2] = OE_C_READ
    ops["key"][f_no + 2] = dist[is_no] * OE_CUSTOMERS + cust[is_no]
    # NewOrder lines
    lines = np.arange(OE_MAX_LINES)
    present = lines[None, :] < ol_cnt[:, None]
    i_pos = (f_no[:, None] + 3 + 2 * lines[None, :])[present]
    s_pos = i_pos + 1
    ops["kind"][i_pos] = OE_I_READ
    ops["key"][i_pos] = items[present]
    ops["kind"][s_pos] = OE_S_NEWORDER
    ops["key"][s_pos] = supply[present] * OE_ITEMS + items[present]
    operands[s_pos, 0] = qty[present]
    operands[s_pos, 1] = (supply != w_no[:, None])[present]
    # Payment ops
    f_p = first[~is_no]
    ops["kind"][f_p] = OE_W_PAY
    ops["key"][f_p] = w_pay
    ops["kind"][f_p + 1] = OE_D_PAY
    ops["key"][f_p + 1] = w_pay * OE_DISTRICTS + d_pay
    ops["kind"][f_p + 2] = OE_C_PAY
    ops["key"][f_p + 2] = (c_w * OE_DISTRICTS + c_d) * OE_CUSTOMERS + c_pay
    for k in range(3):
        operands[f_p + k, 0] = h
    if by_name_frac > 0 and n_pay:
        by_name = rng.random(n_pay) < by_name_frac
        c_run = int(rng.integers(0, 256))
        name = nurand(rng, 255, 0, OE_LAST_NAMES - 1, c_run, n_pay)
        pos = f_p[by_name] + 2
        ops["kind"][pos] = OE_C_PAY_BY_NAME
        ops["key"][pos] = (c_w * OE_DISTRICTS + c_d)[by_name]
        ops["aux"][pos] = name[by_name]
    return KVBatch(txns=txns, ops=ops, operands=operands)


def oe_order_cap(batches, W: int, margin: int = 16) -> int:
    """Order slots per district that hold the initial orders plus every
    NewOrder of ``batches`` even if all of them hit one district."""
    per = np.zeros(W * OE_DISTRICTS, dtype=np.int64)
    for b in batches:
        no = b.txns["type"] == TXN_NEW_ORDER
        dist = b.ops["key"][b.txns["first_op"][no].astype(np.int64) + 1]
        per += np.bincount(dist, minlength=per.size)
    return int(OE_INITIAL_ORDERS + per.max() + margin) if per.size else OE_INITIAL_ORDERS


def order_entry(seed: int = SEEDS[2], W: int = 8, n_txns: int = 1 << 18, order_cap=None,
                by_name_frac: float = 0.0):
    """Initial database, batch and order capacity for the order-entry mix."""
    batch = oe_batch(derive_seed(seed, 40 + W), W, n_txns, by_name_frac=by_name_frac)
    cap = order_cap or oe_order_cap([batch], W)
    return oe_initial_db(seed, W, cap), batch, cap


# ---------------------------------------------------------------------------
# batched form: many independent key-value databases
# ---------------------------------------------------------------------------
def batched_kv(seed: int = SEEDS[3], n_db: int = 64, rec_bits=(16, 22), txn_range=(1000, 262144),
               ops_range=(4, 64), theta: float = 0.8, nfields: int = 8, read_ratio: float = 0.5):
    """``n_db`` databases with 2^U(rec_bits) records (log-uniform sizes) of
    ``nfields`` u64 fields (splitmix64 init), each with one batch whose size
    is log-uniform in ``txn_range`` and whose transactions have a uniform
    number of ops in ``ops_range`` over Zipf(theta) keys.
    Returns a list of (n_records, table, batch)."""
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 51)))
    out = []
    for i in range(n_db):
        bits = int(rng.integers(rec_bits[0], rec_bits[1] + 1))
        nrec = 1 << bits
        n_txns = int(round(math.exp(rng.uniform(math.log(txn_range[0]), math.log(txn_range[1])))))
        s = derive_seed(seed, 1000 + i)
        table = kv_table_splitmix(s, nrec, nfields)
        batch = kv_batch(derive_seed(s, 3), nrec=nrec, nfields=nfields, n_txns=n_txns,
                         ops_range=ops_range, read_ratio=read_ratio, theta=theta, field_bytes=8)
        out.append((nrec, table, batch))
    return out


# ---------------------------------------------------------------------------
# served form: request traces
# ---------------------------------------------------------------------------
def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival offsets (ns, uint64) of an open-loop Poisson process."""
    rng = np.random.Generator(np.random.PCG64(derive_seed(seed, 61)))
    gaps = rng.exponential(1e9 / rate_per_s, size=n)
    return np.cumsum(gaps).astype(np.uint64)


def interleave(batches, lane_of: np.ndarray) -> KVBatch:
    """One trace from per-lane batches: request i is the next transaction of
    batches[lane_of[i]]; its ops are laid out contiguously in trace order."""
    lane_of = np.asarray(lane_of)
    n = lane_of.size
    counts = [int(np.count_nonzero(lane_of == l)) for l in range(len(batches))]
    for l, b in enumerate(batches):
        if b.n_txns < counts[l]:
            raise ValueError("lane %d has too few transactions" % l)
    idx_in_lane = np.zeros(n, dtype=np.int64)
    for l in range(len(batches)):
        sel = lane_of == l
        idx_in_lane[sel] = np.arange(counts[l])
    txns = np.zeros(n, dtype=TXN_DTYPE)
    src_first = np.zeros(n, dtype=np.int64)
    nops = np.zeros(n, dtype=np.int64)
    for l, b in enumerate(batches):
        sel = lane_of == l
        t = b.txns[idx_in_lane[sel]]
        src_first[sel] = t["first_op"]
        nops[sel] = t["n_ops"]
        txns["type"][sel] = t["type"]
    txns["n_ops"] = nops
    first = np.zeros(n, dtype=np.int64)
    if n:
        first[1:] = np.cumsum(nops)[:-1]
    txns["first_op"] = first
    total = int(nops.sum())
    ops = np.zeros(total, dtype=OP_DTYPE)
    operands = np.zeros((total, 2), dtype=np.uint64)
    rep = np.repeat(np.arange(n), nops)
    within = np.arange(total) - np.repeat(first, nops)
    src = np.repeat(src_first, nops) + within
    for l, b in enumerate(batches):
        sel = lane_of[rep] == l
        ops[sel] = b.ops[src[sel]]
        operands[sel] = b.operands[src[sel]]
    return KVBatch(txns=txns, ops=ops, operands=operands)


def select(batch: KVBatch, idx) -> KVBatch:
    """The transactions ``idx`` of ``batch`` (in that order) as a batch of
    their own."""
    idx = np.asarray(idx, dtype=np.int64)
    t = batch.txns[idx]
    nops = t["n_ops"].astype(np.int64)
    first = np.zeros(idx.size, dtype=np.int64)
    if idx.size:
        first[1:] = np.cumsum(nops)[:-1]
    src = np.repeat(t["first_op"].astype(np.int64), nops) + \
        (np.arange(int(nops.sum())) - np.repeat(first, nops))
    txns = t.copy()
    txns["first_op"] = first
    return KVBatch(txns=txns, ops=batch.ops[src].copy(), operands=batch.operands[src].copy())


def disjoint_kv(seed: int, n_txns: int, nrec: int, nfields: int, ops_per_txn: int = 16,
                read_ratio: float = 0.8) -> KVBatch:
    """Transactions on pairwise disjoint keys: request r uses keys
    [r * ops_per_txn, (r + 1) * ops_per_txn)."""
    if n_txns * ops_per_txn > nrec:
        raise ValueError("not enough records for disjoint transactions")
    b = kv_batch(seed, nrec=nrec, nfields=nfields, n_txns=n_txns, ops_per_txn=ops_per_txn,
                 read_ratio=read_ratio, theta=0.0)
    b.ops["key"] = np.arange(n_txns * ops_per_txn, dtype=np.uint32)
    return b
