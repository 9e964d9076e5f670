"""GPU parity of OCC with group commit (key-value batches) against the oracle.

Group commit runs the transactions that share a most-written record as one
unit; every member's outcome must still be the serial execution in the
reported commit order: the oracle replays every committed history from the
same initial table, every read value and every word of the final table bit
for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2406_10158_gb300 import workload as wl

pytestmark = pytest.mark.gpu

HOT = {"backoff_cap_ns": 16_000_000}


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine
    return engine


def run_gc(eng, db, batch, group, min_writes=2, timeout_s=120, **kw):
    p = eng.params(group_commit=group, group_min_writes=min_writes, **kw)
    return db.run("occ", batch, p, timeout_s=timeout_s)


def check(table, final, batch, res, reads, stats, require_all=True):
    rep = oracle.replay_check(table, final, batch, res, reads, require_all=require_all)
    assert rep["ok"], (rep, stats)
    return rep


def launches_of(db):
    return db.stage_history(1)[-1]["kernel_launches"]


@pytest.mark.parametrize("group", [2, 4, 8])
@pytest.mark.parametrize("lanes", [2, 4, 16, 32])
def test_group_commit_replays(eng, group, lanes):
    """Hot keys (Zipf 0.9 over 8,192 records), ragged op counts 1..16, unit
    sizes and lane-group widths (narrow groups stage a unit per few lanes: one
    warp per block keeps the block's staging within an SM's shared memory):
    the committed history replays exactly, and the unit formation ran (more
    launches than plain OCC)."""
    warps = 1 if lanes <= 4 else 4
    nrec = 8192
    table = wl.kv_table_splitmix(41, nrec, 4)
    batch = wl.kv_batch(700 + group * 10 + lanes, nrec=nrec, nfields=4, n_txns=8192,
                        ops_range=(1, 16), read_ratio=0.5, theta=0.9)
    with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8, max_ops_per_txn=16,
                      max_batch_txns=8192) as db:
        db.load_kv(table)
        _, _, _ = db.run("occ", batch, eng.params(lanes_per_txn=lanes, warps_per_block=warps,
                                                  **HOT))
        plain = launches_of(db)
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, batch, group, lanes_per_txn=lanes,
                                   warps_per_block=warps, **HOT)
        assert launches_of(db) > plain
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, stats)


@pytest.mark.parametrize("group", [2, 8])
def test_group_commit_sixteen_byte_slots(eng, group):
    """16-byte slots (u64 lane plus a u16 lane) under Zipf 0.99."""
    nrec = 4096
    table = wl.kv_table_bytes(43, nrec, 3)
    batch = wl.kv_batch(51 + group, nrec=nrec, nfields=3, n_txns=6000, ops_per_txn=8,
                        read_ratio=0.5, theta=0.99, field_bytes=16)
    with eng.Database("kv", n_records=nrec, n_fields=3, field_bytes=16, max_ops_per_txn=8,
                      max_batch_txns=6000) as db:
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, batch, group, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, stats)


def test_group_commit_one_record_for_everyone(eng):
    """Every transaction writes record 0, on varying fields, and reads or
    writes a few others (some of them shared): units of 8 compose the record's
    fields in commit order; the readers of record 0 inside a unit see the
    writes of the members before them."""
    rng = np.random.default_rng(5)
    txns = []
    for t in range(3000):
        ops = [(0, int(rng.integers(0, 3)), 1, int(rng.integers(-50, 50)), 0)]
        others = rng.choice(np.arange(1, 40), size=int(rng.integers(0, 5)), replace=False)
        for k in others:
            ops.append((int(k), int(rng.integers(0, 3)), int(rng.integers(0, 2)),
                        int(rng.integers(-9, 9)), 0))
        rng.shuffle(ops)
        txns.append(ops)
    # readers of record 0 among them
    for t in range(0, 3000, 7):
        k, f, _, _, _ = txns[t][0]
        txns[t] = [(0, 1, 0, 0, 0)] + [o for o in txns[t] if o[0] != 0]
    batch = wl.kv_batch_from_lists(txns)
    table = wl.kv_table_splitmix(3, 64, 3)
    with eng.Database("kv", n_records=64, n_fields=3, field_bytes=8, max_ops_per_txn=8,
                      max_batch_txns=3000) as db:
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, batch, 8, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, stats)


def test_group_commit_invalid_members(eng):
    """Malformed transactions inside units come back INVALID and the other
    members of their units commit; the empty and read-only batches behave as
    under plain OCC."""
    with eng.Database("kv", n_records=64, n_fields=2, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=64) as db:
        table = wl.kv_table_splitmix(1, 64, 2)
        db.load_kv(table)
        empty = wl.kv_batch_from_lists([])
        res, reads, stats = run_gc(eng, db, empty, 4)
        assert stats["committed"] == 0 and res.size == 0
        ro = wl.kv_batch(2, nrec=64, nfields=2, n_txns=16, ops_per_txn=4, read_ratio=1.0)
        res, reads, stats = run_gc(eng, db, ro, 4)
        assert np.array_equal(db.read_kv(), table)
        assert np.array_equal(reads[:, 0], table[ro.ops["field"], ro.ops["key"]])
        lists = []
        for t in range(24):
            if t % 5 == 1:
                lists.append([(7, 0, 1, 3, 0), (7, 1, 0, 0, 0)])        # duplicate key
            elif t % 5 == 3:
                lists.append([(7, 0, 1, 3, 0), (64, 0, 0, 0, 0)])       # key out of range
            else:
                lists.append([(7, t % 2, 1, t + 1, 0), (9 + t % 3, 0, t % 2, 2, 0)])
        bad = wl.kv_batch_from_lists(lists)
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, bad, 4)
        final = db.read_kv()
        want_bad = [t % 5 in (1, 3) for t in range(24)]
        assert (res["status"][want_bad] == oracle.ST_INVALID).all()
        assert (res["status"][~np.array(want_bad)] == oracle.ST_COMMITTED).all()
        assert stats["invalid"] == sum(want_bad)
        check(table, final, bad, res, reads, stats, require_all=False)


def test_group_commit_zipf_099_finishes(eng):
    """Zipf 0.99: most writers of the hottest record touch other contended
    records too, so few units form; the batch commits in full (units that
    keep failing take turns through the retry queues) and replays exactly."""
    nrec = 1 << 14
    table = wl.kv_table_splitmix(12, nrec, 4)
    batch = wl.kv_batch(13, nrec=nrec, nfields=4, n_txns=16384, ops_per_txn=8,
                        read_ratio=0.5, theta=0.99)
    with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8, max_ops_per_txn=8,
                      max_batch_txns=16384) as db:
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, batch, 8, min_writes=16, lanes_per_txn=32,
                                   timeout_s=300)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, stats)


def test_group_commit_injected_aborts(eng):
    """Forced aborts of single members at the commit point (30%): the other
    members commit, the aborted ones retry, the history replays exactly."""
    nrec = 2048
    table = wl.kv_table_splitmix(77, nrec, 4)
    batch = wl.kv_batch(78, nrec=nrec, nfields=4, n_txns=4096, ops_per_txn=8,
                        read_ratio=0.5, theta=0.95)
    with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8, max_ops_per_txn=8,
                      max_batch_txns=4096) as db:
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, batch, 8, inject_abort_ppm=300000,
                                   backoff_base_ns=200, backoff_cap_ns=20000, seed=99)
        final = db.read_kv()
    assert stats["aborts"] > 0.2 * batch.n_txns, stats
    assert (res["attempts"] > 1).any()
    check(table, final, batch, res, reads, stats)


def test_group_commit_attempt_budget(eng):
    """Every attempt forced to abort, a budget of 3 attempts: every member ends
    TIMEOUT after exactly 3 attempts, nothing is left locked, and the next
    batch on the database runs normally."""
    nrec = 512
    table = wl.kv_table_splitmix(8, nrec, 2)
    batch = wl.kv_batch(9, nrec=nrec, nfields=2, n_txns=512, ops_per_txn=4, read_ratio=0.3,
                        theta=0.99)
    with eng.Database("kv", n_records=nrec, n_fields=2, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=512) as db:
        db.load_kv(table)
        res, reads, stats = run_gc(eng, db, batch, 8, inject_abort_ppm=1000000, max_attempts=3)
        assert (res["status"] == oracle.ST_TIMEOUT).all()
        assert (res["attempts"] == 3).all()
        assert "attempts" in stats["errors"]
        assert np.array_equal(db.read_kv(), table)
        res, reads, stats = run_gc(eng, db, batch, 8, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, stats)


@pytest.mark.slow
@pytest.mark.parametrize("theta", [0.8, 0.99])
def test_group_commit_full_size(eng, theta):
    """The key-value sweep's workload (2^24 records x 10 fields in 16-byte
    slots, 2^20 txns x 16 ops, read ratio 0.5) with units of 4 and 8, each
    batch replayed in full."""
    table, batch = wl.ycsb_kv(theta=theta, read_ratio=0.5)
    state = table
    with eng.Database("kv", n_records=1 << 24, n_fields=10, field_bytes=16,
                      max_batch_txns=1 << 20) as db:
        db.load_kv(state)
        for group in (4, 8):
            res, reads, stats = run_gc(eng, db, batch, group, min_writes=32, timeout_s=300)
            final = db.read_kv()
            assert stats["committed"] == batch.n_txns, (group, stats)
            rep = oracle.replay_check(state, final, batch, res, reads)
            assert rep["ok"], (group, rep)
            state = final
