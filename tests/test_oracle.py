"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself: a golden
fixture worked by hand, closed forms (a single hot record's reads are the
prefix sums of the deltas in commit order), the read-only and disjoint special
cases, conservation of the table sum, brute force over every serial order, and
the published first outputs of splitmix64.  ``test_mutants_are_caught``
plants plausible mistakes in a copy of oracle.c and checks that some pin fails
for each one.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2406_10158_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _golden_batch(g):
    lists = [[(k, f, kind, d & M64, 0) for (k, f, kind, d) in t] for t in g["txns"]]
    return wl.kv_batch_from_lists(lists)


def _golden_table(g):
    return np.array(g["table"]["values"], dtype=np.uint64)


# ---------------------------------------------------------------------------
# pins, each usable with an alternative oracle build (see the mutant test)
# ---------------------------------------------------------------------------
def pin_golden_serial_orders(lib):
    g = _golden("kv_three_txns.json")
    batch, table = _golden_batch(g), _golden_table(g)
    for key, exp in g["serial"].items():
        order = [int(x) for x in key.split(",")]
        fin, reads = oracle.serial(table, batch, order=order, lib=lib)
        got = reads[:, 0].reshape(3, 2).tolist()
        assert got == exp["reads"], (key, got)
        assert fin[0].tolist() == exp["final"], (key, fin)


def pin_golden_brute_force(lib):
    g = _golden("kv_three_txns.json")
    batch, table = _golden_batch(g), _golden_table(g)
    for key, exp in g["serial"].items():
        reads = np.zeros((6, 2), dtype=np.uint64)
        reads[:, 0] = np.array(exp["reads"], dtype=np.uint64).ravel()
        fin = np.array([exp["final"]], dtype=np.uint64)
        n, first = oracle.brute_force(table, batch, fin, reads, lib=lib)
        assert n == 1 and ",".join(map(str, first)) == key, (key, n, first)
    bad = g["not_serializable"]
    reads = np.zeros((6, 2), dtype=np.uint64)
    reads[:, 0] = np.array(bad["reads"], dtype=np.uint64).ravel()
    n, _ = oracle.brute_force(table, batch, np.array([bad["final"]], dtype=np.uint64),
                              reads, lib=lib)
    assert n == 0


def pin_hot_key_prefix_sums(lib, field_bytes=8):
    """n transactions each ADD to record (3, field 1): the read values are the
    initial value plus the prefix sums of the deltas in execution order."""
    rng = np.random.default_rng(5)
    n, nrec, nf = 40, 8, 2
    deltas = [int(x) for x in rng.integers(-(1 << 62), 1 << 62, size=n)]
    his = [int(x) for x in rng.integers(0, 1 << 16, size=n)]
    lists = [[(3, 1, wl.OP_ADD, d & M64, h if field_bytes == 16 else 0),
              (5, 0, wl.OP_READ, 0, 0)] for d, h in zip(deltas, his)]
    batch = wl.kv_batch_from_lists(lists)
    if field_bytes == 8:
        table = rng.integers(0, 1 << 63, size=(nf, nrec), dtype=np.uint64)
    else:
        table = rng.integers(0, 1 << 63, size=(nf, nrec, 2), dtype=np.uint64)
        table[..., 1] &= np.uint64(0xFFFF)
    order = rng.permutation(n)
    fin, reads = oracle.serial(table, batch, order=order, lib=lib)
    lo = int(table[1, 3] if field_bytes == 8 else table[1, 3, 0])
    hi = 0 if field_bytes == 8 else int(table[1, 3, 1])
    for t in order:
        assert int(reads[2 * t, 0]) == lo
        assert int(reads[2 * t, 1]) == hi
        assert int(reads[2 * t + 1, 0]) == int(table[0, 5] if field_bytes == 8 else table[0, 5, 0])
        lo = (lo + deltas[t]) & M64
        if field_bytes == 16:
            hi = (hi + his[t]) & 0xFFFF
    if field_bytes == 8:
        assert int(fin[1, 3]) == lo
    else:
        assert int(fin[1, 3, 0]) == lo and int(fin[1, 3, 1]) == hi
    untouched = np.ones(fin.shape[:2], dtype=bool)
    untouched[1, 3] = False
    assert np.array_equal(fin[untouched], table[untouched])


def pin_hot_key_16(lib):
    pin_hot_key_prefix_sums(lib, field_bytes=16)


def pin_read_only_batch(lib):
    """A batch of READs returns the initial values (the splitmix64 closed form)
    and leaves the table unchanged."""
    seed = 1234
    table = wl.kv_table_splitmix(seed, 512, 8)
    batch = wl.kv_batch(9, nrec=512, nfields=8, n_txns=64, ops_per_txn=16, read_ratio=1.0)
    fin, reads = oracle.serial(table, batch, lib=lib)
    assert np.array_equal(fin, table)
    expect = wl.splitmix64_init(seed, batch.ops["key"], batch.ops["field"], 8)
    assert np.array_equal(reads[:, 0], expect)
    assert not reads[:, 1].any()


def pin_disjoint_order_independent(lib):
    """Transactions on disjoint keys give the same outcome in any order."""
    rng = np.random.default_rng(3)
    keys = rng.permutation(256)[: 16 * 8].reshape(16, 8)
    lists = [[(int(k), int(rng.integers(0, 4)), int(rng.integers(0, 2)),
               int(rng.integers(0, 1 << 63)), 0) for k in row] for row in keys]
    batch = wl.kv_batch_from_lists(lists)
    table = rng.integers(0, 1 << 63, size=(4, 256), dtype=np.uint64)
    f1, r1 = oracle.serial(table, batch, order=np.arange(16), lib=lib)
    f2, r2 = oracle.serial(table, batch, order=rng.permutation(16), lib=lib)
    assert np.array_equal(f1, f2) and np.array_equal(r1, r2)
    assert not np.array_equal(f1, table)


def _numpy_sum(table):
    lo = table if table.ndim == 2 else table[..., 0]
    s0 = int(np.sum(lo, dtype=np.uint64))
    s1 = 0 if table.ndim == 2 else int(np.sum(table[..., 1] & np.uint64(0xFFFF),
                                              dtype=np.uint64)) & 0xFFFF
    return s0, s1


def pin_conservation(lib):
    """Sum of the table after = before + sum of the ADD deltas (per lane)."""
    for fb in (8, 16):
        rng = np.random.default_rng(11 + fb)
        if fb == 8:
            table = wl.kv_table_splitmix(77, 1000, 4)
        else:
            table = wl.kv_table_bytes(77, 1000, 4)
        batch = wl.kv_batch(21, nrec=1000, nfields=4, n_txns=300, ops_per_txn=8,
                            read_ratio=0.4, theta=0.9, field_bytes=fb)
        fin, _ = oracle.serial(table, batch, order=rng.permutation(300), lib=lib)
        add = batch.ops["kind"] == wl.OP_ADD
        d0 = int(np.sum(batch.operands[add, 0], dtype=np.uint64))
        d1 = int(np.sum(batch.operands[add, 1], dtype=np.uint64)) & 0xFFFF
        b0, b1 = _numpy_sum(table)
        a0, a1 = _numpy_sum(fin)
        assert a0 == (b0 + d0) & M64
        assert a1 == (b1 + d1) & 0xFFFF
        assert oracle.table_sum(fin, lib=lib) == (a0, a1)


def pin_byte_lanes(lib):
    """16-byte slot: lane 0 wraps mod 2^64 without carrying into lane 1; bytes
    8-9 wrap mod 2^16; bytes 10-15 are untouched; the read is the old slot."""
    table = np.zeros((1, 2, 2), dtype=np.uint64)
    table[0, 1] = (M64, 0x0000ABCD0000FFFF)
    batch = wl.kv_batch_from_lists([[(1, 0, wl.OP_ADD, 1, 1)]])
    fin, reads = oracle.serial(table, batch, lib=lib)
    assert [int(x) for x in fin[0, 1]] == [0, 0x0000ABCD00000000]
    assert [int(x) for x in reads[0]] == [M64, 0x0000ABCD0000FFFF]


def pin_replay_accepts_true_order_rejects_swap(lib):
    """Replaying in the order that produced an outcome matches it; swapping two
    transactions that conflict on a record is detected."""
    table = wl.kv_table_splitmix(5, 64, 2)
    batch = wl.kv_batch(6, nrec=64, nfields=2, n_txns=50, ops_per_txn=6, read_ratio=0.5)
    rng = np.random.default_rng(0)
    order = rng.permutation(50)
    fin, reads = oracle.serial(table, batch, order=order, lib=lib)
    res = np.zeros(50, dtype=wl.RESULT_DTYPE)
    res["status"] = oracle.ST_COMMITTED
    res["commit_order"][order] = np.arange(50)
    rep = oracle.replay_check(table, fin, batch, res, reads, lib=lib)
    assert rep["ok"], rep
    # find two adjacent txns in `order` that both ADD to a common record
    keys = batch.ops["key"].reshape(50, 6)
    adds = batch.ops["kind"].reshape(50, 6) == wl.OP_ADD
    for i in range(49):
        a, b = order[i], order[i + 1]
        if set(keys[a][adds[a]]) & set(keys[b][adds[b]]):
            swapped = res.copy()
            swapped["commit_order"][a], swapped["commit_order"][b] = i + 1, i
            rep2 = oracle.replay_check(table, fin, batch, swapped, reads, lib=lib)
            assert not rep2["ok"] and rep2["n_read_mismatch"] > 0
            break
    else:
        pytest.fail("no adjacent conflicting pair")


def pin_brute_force_random_tiny(lib):
    """For random batches of <= 6 transactions on a few hot records, the serial
    outcome of a random order is found by brute force, and the first matching
    order reproduces it."""
    rng = np.random.default_rng(42)
    for trial in range(20):
        n = int(rng.integers(2, 7))
        lists = []
        for _ in range(n):
            ks = rng.permutation(4)[: int(rng.integers(1, 4))]
            lists.append([(int(k), 0, int(rng.integers(0, 2)), int(rng.integers(1, 1000)), 0)
                          for k in ks])
        batch = wl.kv_batch_from_lists(lists)
        table = rng.integers(0, 1000, size=(1, 4), dtype=np.uint64)
        order = rng.permutation(n)
        fin, reads = oracle.serial(table, batch, order=order, lib=lib)
        m, first = oracle.brute_force(table, batch, fin, reads, lib=lib)
        assert m >= 1
        f2, r2 = oracle.serial(table, batch, order=first, lib=lib)
        assert np.array_equal(f2, fin) and np.array_equal(r2, reads)


def _tiny_oe(lib):
    W, cap = 1, 3016
    db = wl.oe_initial_db(7, W, cap)
    return W, cap, db


def pin_oe_stock_rule_golden(lib):
    """A NewOrder with five lines whose stock levels and quantities are the
    hand-worked cases of the golden fixture."""
    g = _golden("oe_stock_and_payment.json")
    W, cap, db = _tiny_oe(lib)
    items = [11, 22, 33, 44, 55]
    for it, case, price in zip(items, g["stock_cases"], g["prices"]):
        db["s_quantity"][it] = case["old"]
        db["i_price"][it] = price
    ops = [(0, wl.OE_W_READ, 0, 0), (4, wl.OE_D_NEWORDER, 0, 0), (4 * 3000 + 17, wl.OE_C_READ, 0, 0)]
    for it, case in zip(items, g["stock_cases"]):
        ops += [(it, wl.OE_I_READ, 0, 0), (it, wl.OE_S_NEWORDER, case["qty"], 0)]
    batch = _oe_batch_from_lists([(wl.TXN_NEW_ORDER, ops)])
    fin, reads = oracle.oe_serial(db, W, cap, batch, lib=lib)
    for l, (it, case) in enumerate(zip(items, g["stock_cases"])):
        assert fin["s_quantity"][it] == case["new"], (case, fin["s_quantity"][it])
        assert fin["s_ytd"][it] == case["qty"]
        assert fin["s_order_cnt"][it] == 1
        assert int(reads[4 + 2 * l, 0]) == case["old"]
        assert int(reads[3 + 2 * l, 0]) == g["prices"][l]
    assert int(reads[1, 0]) == 3001 and fin["d_next_o_id"][4] == 3002
    slot = 4 * cap + 3000
    assert fin["o_ol_cnt"][slot] == 5 and fin["o_c_id"][slot] == 17
    assert fin["no_flag"][slot] == 1 and fin["o_all_local"][slot] == 1
    amounts = fin["ol_amount"][slot * 15: slot * 15 + 5].tolist()
    assert amounts == g["amounts"]
    assert fin["ol_quantity"][slot * 15 + 5] == 0
    assert oracle.oe_consistency(fin, W, cap, lib=lib) == 0


def pin_oe_payment_golden(lib):
    g = _golden("oe_stock_and_payment.json")["payment"]
    W, cap, db = _tiny_oe(lib)
    b = g["before"]
    db["w_ytd"][0] = b["w_ytd"]
    db["d_ytd"][:] = 0
    db["d_ytd"][3] = b["d_ytd"]
    db["w_ytd"][0] = b["w_ytd"]
    cust = 3 * 3000 + 99
    for c in ("c_balance", "c_ytd_payment", "c_payment_cnt"):
        db[c][cust] = b[c]
    h = g["h"]
    batch = _oe_batch_from_lists([(wl.TXN_PAYMENT, [(0, wl.OE_W_PAY, h, 0),
                                                     (3, wl.OE_D_PAY, h, 0),
                                                     (cust, wl.OE_C_PAY, h, 0)])])
    fin, reads = oracle.oe_serial(db, W, cap, batch, lib=lib)
    a = g["after"]
    assert fin["w_ytd"][0] == a["w_ytd"] and fin["d_ytd"][3] == a["d_ytd"]
    for c in ("c_balance", "c_ytd_payment", "c_payment_cnt"):
        assert fin[c][cust] == a[c], c
    assert [int(reads[0, 0]), int(reads[1, 0])] == [b["w_ytd"], b["d_ytd"]]
    assert reads[2].view(np.int64).tolist() == [b["c_balance"], b["c_payment_cnt"]]


def pin_oe_invariants(lib):
    """After a random mix run serially in a random order: the consistency
    conditions hold, stock year-to-date grows by the ordered quantity, the
    warehouses' year-to-date grows by the paid amounts, and the order lines
    inserted equal the lines ordered."""
    W = 2
    db, batch, cap = wl.order_entry(seed=99, W=W, n_txns=3000)
    order = np.random.default_rng(1).permutation(batch.n_txns)
    fin, _ = oracle.oe_serial(db, W, cap, batch, order=order, lib=lib)
    assert oracle.oe_consistency(fin, W, cap, lib=lib) == 0
    s_ops = batch.ops["kind"] == wl.OE_S_NEWORDER
    assert fin["s_ytd"].sum() - db["s_ytd"].sum() == int(batch.operands[s_ops, 0].sum())
    assert fin["s_order_cnt"].sum() - db["s_order_cnt"].sum() == int(s_ops.sum())
    n_remote = int(batch.operands[s_ops, 1].sum())
    assert n_remote > 0
    assert fin["s_remote_cnt"].sum() - db["s_remote_cnt"].sum() == n_remote
    pay = batch.ops["kind"] == wl.OE_W_PAY
    paid = int(batch.operands[pay, 0].sum())
    assert fin["w_ytd"].sum() - db["w_ytd"].sum() == paid
    assert db["c_balance"].sum() - fin["c_balance"].sum() == paid
    new_lines = np.count_nonzero(fin["ol_quantity"]) - np.count_nonzero(db["ol_quantity"])
    assert new_lines == int(s_ops.sum())
    no = batch.txns["type"] == wl.TXN_NEW_ORDER
    assert fin["d_next_o_id"].sum() - db["d_next_o_id"].sum() == int(no.sum())


def _oe_consistent_db(lib):
    """A consistent order-entry database: a random mix run serially."""
    W = 2
    db, batch, cap = wl.order_entry(seed=99, W=W, n_txns=3000)
    order = np.random.default_rng(1).permutation(batch.n_txns)
    fin, _ = oracle.oe_serial(db, W, cap, batch, order=order, lib=lib)
    return W, cap, db, batch, order, fin


def pin_oe_consistency_flags_each_violation(lib):
    """The consistency check reports each of its three conditions by its own
    bit and nothing else: a district whose next order id is one past its
    newest order (bit 1), a warehouse whose year-to-date differs from the sum
    of its districts' (bit 2), and an order line present beyond its order's
    line count (bit 4)."""
    W, cap, _, _, _, fin = _oe_consistent_db(lib)
    assert oracle.oe_consistency(fin, W, cap, lib=lib) == 0

    bad = {c: a.copy() for c, a in fin.items()}
    bad["d_next_o_id"][7] += 1
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 1

    bad = {c: a.copy() for c, a in fin.items()}
    bad["d_next_o_id"][3] -= 1
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 1

    bad = {c: a.copy() for c, a in fin.items()}
    bad["w_ytd"][1] += 1
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 2

    bad = {c: a.copy() for c, a in fin.items()}
    bad["d_ytd"][4] -= 5            # district 4 belongs to warehouse 0
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 2

    bad = {c: a.copy() for c, a in fin.items()}
    slot = 12 * cap + 5             # an initial order of district 12
    cnt = int(bad["o_ol_cnt"][slot])
    assert 0 < cnt < 15
    bad["ol_quantity"][slot * 15 + cnt] = 3
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 4

    bad = {c: a.copy() for c, a in fin.items()}
    bad["ol_quantity"][slot * 15] = 0   # a line missing inside the count
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 4

    bad = {c: a.copy() for c, a in fin.items()}
    bad["d_next_o_id"][0] += 1
    bad["w_ytd"][0] += 1
    assert oracle.oe_consistency(bad, W, cap, lib=lib) == 3


def pin_oe_replay_rejects_wrong_outcomes(lib):
    """The order-entry replay check accepts the order that produced an
    outcome and rejects: two payments to one district swapped in the commit
    order (their year-to-date reads differ), one flipped read value, and one
    corrupted word of a final column."""
    W, cap, db, batch, order, fin = _oe_consistent_db(lib)
    _, reads = oracle.oe_serial(db, W, cap, batch, order=order, lib=lib)
    res = np.zeros(batch.n_txns, dtype=wl.RESULT_DTYPE)
    res["status"] = oracle.ST_COMMITTED
    res["commit_order"][order] = np.arange(batch.n_txns)
    rep = oracle.oe_replay_check(db, fin, W, cap, batch, res, reads, lib=lib)
    assert rep["ok"] and rep["n_committed"] == batch.n_txns, rep

    # two payments on the same district, adjacent in the commit order
    pay = batch.txns["type"] == wl.TXN_PAYMENT
    dist = batch.ops["key"][batch.txns["first_op"].astype(np.int64) + 1]
    pos = {}
    for i, t in enumerate(order):
        if pay[t]:
            pos.setdefault(int(dist[t]), []).append(i)
    pair = next((p[k], p[k + 1]) for p in pos.values() for k in range(len(p) - 1)
                if p[k + 1] == p[k] + 1)
    swapped = res.copy()
    a, b = order[pair[0]], order[pair[1]]
    swapped["commit_order"][a], swapped["commit_order"][b] = pair[1], pair[0]
    rep = oracle.oe_replay_check(db, fin, W, cap, batch, swapped, reads, lib=lib)
    assert not rep["ok"] and rep["n_read_mismatch"] >= 2, rep

    flipped = reads.copy()
    flipped[17, 0] ^= np.uint64(1)
    rep = oracle.oe_replay_check(db, fin, W, cap, batch, res, flipped, lib=lib)
    assert not rep["ok"] and rep["n_read_mismatch"] == 1, rep

    for col in ("s_quantity", "c_balance", "ol_amount"):
        bad = {c: a.copy() for c, a in fin.items()}
        nz = np.flatnonzero(bad[col] != db[col])
        bad[col][nz[len(nz) // 2]] += 1
        rep = oracle.oe_replay_check(db, bad, W, cap, batch, res, reads, lib=lib)
        assert not rep["ok"] and rep["bad_columns"] == {col: 1}, (col, rep)


def pin_oe_payment_by_name_golden(lib):
    """A payment by last name in district 0 lands on the customer the
    hand-worked fixture selects (the middle one by first name, then index),
    and a name nobody has is refused."""
    g = _golden("oe_last_name.json")
    W, cap, db = _tiny_oe(lib)
    db["c_last"][:] = 500                          # nobody else has a fixture name
    n = len(g["c_last"])
    db["c_last"][:n] = g["c_last"]
    db["c_first"][:n] = g["c_first"]
    for name, want in g["expected"].items():
        batch = _oe_batch_from_lists([(wl.TXN_PAYMENT, [(0, wl.OE_W_PAY, 700, 0),
                                                         (0, wl.OE_D_PAY, 700, 0),
                                                         (0, wl.OE_C_PAY_BY_NAME, 700, 0)])])
        batch.ops["aux"][2] = int(name)
        if want < 0:
            with pytest.raises(oracle.OracleError):
                oracle.oe_serial(db, W, cap, batch, lib=lib)
            continue
        fin, reads = oracle.oe_serial(db, W, cap, batch, lib=lib)
        changed = np.flatnonzero(fin["c_balance"] != db["c_balance"])
        assert changed.tolist() == [want], (name, changed)
        assert fin["c_balance"][want] == db["c_balance"][want] - 700
        assert fin["c_payment_cnt"][want] == db["c_payment_cnt"][want] + 1
        assert reads[2].view(np.int64).tolist() == [int(db["c_balance"][want]),
                                                     int(db["c_payment_cnt"][want])]


def _oe_batch_from_lists(txns):
    n_ops = sum(len(o) for _, o in txns)
    t = np.zeros(len(txns), dtype=wl.TXN_DTYPE)
    ops = np.zeros(n_ops, dtype=wl.OP_DTYPE)
    operands = np.zeros((n_ops, 2), dtype=np.uint64)
    i = 0
    for j, (typ, lst) in enumerate(txns):
        t[j] = (i, len(lst), typ)
        for key, kind, lo, hi in lst:
            ops[i] = (key, 0, kind, 0)
            operands[i] = (lo & M64, hi & M64)
            i += 1
    return wl.KVBatch(txns=t, ops=ops, operands=operands)


PINS = [pin_golden_serial_orders, pin_golden_brute_force, pin_hot_key_prefix_sums,
        pin_hot_key_16, pin_read_only_batch, pin_disjoint_order_independent,
        pin_conservation, pin_byte_lanes, pin_replay_accepts_true_order_rejects_swap,
        pin_brute_force_random_tiny, pin_oe_stock_rule_golden, pin_oe_payment_golden,
        pin_oe_invariants, pin_oe_consistency_flags_each_violation,
        pin_oe_replay_rejects_wrong_outcomes, pin_oe_payment_by_name_golden]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin(oracle.load())


def test_splitmix64_published_outputs():
    # first outputs of splitmix64 seeded with 0, as published with the
    # reference implementation (Vigna, splitmix64.c)
    got = [int(x) for x in wl.splitmix64_at(0, np.arange(1, 4, dtype=np.uint64))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_commit_sequence_rejects_non_permutations():
    res = np.zeros(4, dtype=wl.RESULT_DTYPE)
    res["status"] = oracle.ST_COMMITTED
    res["commit_order"] = [0, 1, 1, 3]
    with pytest.raises(oracle.OracleError):
        oracle.commit_sequence(res)
    res["commit_order"] = [0, 1, 2, 4]
    with pytest.raises(oracle.OracleError):
        oracle.commit_sequence(res)
    res["commit_order"] = [3, 1, 0, 2]
    assert oracle.commit_sequence(res).tolist() == [2, 1, 3, 0]
    res["status"][1] = oracle.ST_TIMEOUT
    res["commit_order"] = [2, 99, 0, 1]
    assert oracle.commit_sequence(res).tolist() == [2, 3, 0]


def test_oracle_rejects_bad_inputs():
    table = np.zeros((2, 4), dtype=np.uint64)
    for op in [(4, 0, 0, 0, 0), (0, 2, 0, 0, 0), (0, 0, 7, 0, 0)]:
        with pytest.raises(oracle.OracleError):
            oracle.serial(table, wl.kv_batch_from_lists([[op]]))


# ---------------------------------------------------------------------------
# planted mistakes: each must make at least one pin fail
# ---------------------------------------------------------------------------
MUTANTS = {
    "add_wrong_sign": ("s[0] = old_lo + operand[0];", "s[0] = old_lo - operand[0];"),
    "hi_lane_dropped": ("uint64_t b89 = (old_hi + operand[1]) & 0xFFFFull;",
                        "uint64_t b89 = old_hi & 0xFFFFull;"),
    "hi_lane_wide": ("uint64_t b89 = (old_hi + operand[1]) & 0xFFFFull;",
                     "uint64_t b89 = (old_hi + operand[1]) & 0xFFFFFull;"),
    "read_after_write": ("    out[0] = old_lo;\n    out[1] = old_hi;\n    return ORC_OK;\n}",
                         "    out[0] = s[0];\n    out[1] = old_hi;\n    return ORC_OK;\n}"),
    "layout_transposed": ("((uint64_t)field * db->nrec + key) * words",
                          "((uint64_t)key * db->nfields + field) * words"),
    "replay_reversed": ("const orc_txn *t = &txns[order[k]];",
                        "const orc_txn *t = &txns[order[nc - 1 - k]];"),
    "stock_boundary": ("if (q >= qty + 10)", "if (q > qty + 10)"),
    "stock_refill": ("db->s_quantity[k] = q - qty + 91;", "db->s_quantity[k] = q - qty + 90;"),
    "balance_sign": ("db->c_balance[k] -= h;", "db->c_balance[k] += h;"),
    "amount_no_price": ("db->ol_amount[ol] = qty * price;", "db->ol_amount[ol] = qty;"),
    "no_next_o_id": ("db->d_next_o_id[k] += 1;", "db->d_next_o_id[k] += 0;"),
    "remote_ignored": ("db->s_remote_cnt[k] += remote;", "db->s_remote_cnt[k] += 0;"),
    "consistency_always_ok": ("    return bad;\n}", "    return 0;\n}"),
    "consistency_no_next_o_id": ("            bad |= 1;", "            bad |= 0;"),
    "consistency_no_ytd_sum": ("if (s != db->w_ytd[w]) bad |= 2;", "if (s != db->w_ytd[w]) bad |= 0;"),
    "consistency_no_lines": ("if (present != (l < cnt)) bad |= 4;", "if (present != (l < cnt)) bad |= 0;"),
    "consistency_lines_off_by_one": ("if (present != (l < cnt)) bad |= 4;",
                                     "if (present != (l <= cnt)) bad |= 4;"),
    "by_name_upper_middle": ("int64_t want = (n + 1) / 2 - 1;", "int64_t want = n / 2;"),
    "by_name_ties_descending": ("(db->c_first[base + o] == db->c_first[base + c] && o < c))",
                                "(db->c_first[base + o] == db->c_first[base + c] && o > c))"),
    "by_name_ignores_first": ("if (db->c_first[base + o] < db->c_first[base + c] ||",
                              "if (0 ||"),
    "oe_insert_wrong_slot": ("uint64_t slot = (uint64_t)dist * db->order_cap + (uint64_t)(o_id - 1);",
                             "uint64_t slot = (uint64_t)dist * db->order_cap + (uint64_t)o_id;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants_are_caught(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    (tmp_path / "oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(os.path.dirname(oracle.__file__), "oracle.h"), tmp_path)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-o", str(so),
                    str(tmp_path / "oracle.c")], check=True)
    lib = oracle.load(str(so))
    failed = []
    for pin in PINS:
        try:
            pin(lib)
        except (AssertionError, oracle.OracleError):
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"


# ---------------------------------------------------------------------------
# payment by last name: the selection rule (a reading; the kernel is not built)
# ---------------------------------------------------------------------------
def _last_name_golden():
    with open(os.path.join(GOLDEN, "oe_last_name.json")) as f:
        g = json.load(f)
    return g["c_last"], g["c_first"], {int(k): v for k, v in g["expected"].items()}


def test_customer_by_last_name_golden():
    last, first, expected = _last_name_golden()
    for name, want in expected.items():
        assert oracle.customer_by_last_name(last, first, name) == want, name


def test_customer_by_last_name_golden_rejects_plausible_mistakes():
    """Each plausible misreading of the rule disagrees with the hand-worked
    fixture somewhere: the upper middle, ties by descending index, no
    first-name order at all, and counting from zero."""
    last, first, expected = _last_name_golden()

    def pick(order, position):
        def f(name):
            named = [c for c in range(len(last)) if last[c] == name]
            if not named:
                return -1
            return order(named)[position(len(named))]
        return f

    by_first = lambda named: sorted(named, key=lambda c: (first[c], c))
    variants = {
        "upper middle": pick(by_first, lambda n: n // 2),
        "ties by descending index": pick(lambda named: sorted(named, key=lambda c: (first[c], -c)),
                                         lambda n: (n + 1) // 2 - 1),
        "index order": pick(sorted, lambda n: (n + 1) // 2 - 1),
        "zero-based ceil": pick(by_first, lambda n: min((n + 1) // 2, n - 1)),
    }
    for label, f in variants.items():
        assert any(f(name) != want for name, want in expected.items()), label


def test_customer_by_last_name_on_generated_districts():
    names = wl.oe_customer_names(5, 1)
    last = names["c_last"].reshape(wl.OE_DISTRICTS, wl.OE_CUSTOMERS)
    first = names["c_first"].reshape(wl.OE_DISTRICTS, wl.OE_CUSTOMERS)
    rng = np.random.default_rng(0)
    for d in range(2):
        for name in rng.integers(0, wl.OE_LAST_NAMES, size=20):
            c = oracle.customer_by_last_name(last[d], first[d], int(name))
            named = np.nonzero(last[d] == name)[0]
            assert c in named                                  # every name exists
            key = lambda i: (int(first[d][i]), int(i))
            before = sum(key(i) < key(c) for i in named)
            assert before == (named.size + 1) // 2 - 1
