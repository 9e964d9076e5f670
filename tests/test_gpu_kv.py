"""GPU parity of the key-value path against the CPU oracle.

Every committed history the engine reports is replayed by the oracle in the
reported commit order from the same initial table; every read value and every
word of the final table must match bit for bit.  The deterministic scheme must
in addition equal serial execution in transaction-id order.
"""
import numpy as np
import pytest

import oracle
from paper_2406_10158_gb300 import workload as wl

pytestmark = pytest.mark.gpu
SCHEMES = ["occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc", "det", "det-dataflow", "det-gacco"]


# Under heavy contention no-wait locking and timestamp ordering need retry
# windows of milliseconds (thousands of contenders x microseconds per hold).
HOT = {"backoff_cap_ns": 16_000_000}


def go(eng, db, scheme, batch, timeout_s=120, **kw):
    """Run a batch; "det-dataflow" is the deterministic scheme run op by op
    (key-value batches otherwise take the prefix-sum evaluation), "det-gacco"
    the same with every access to a record ordered, reads included."""
    if scheme == "det-dataflow":
        scheme, kw = "det", dict(kw, det_dataflow=1)
    elif scheme == "det-gacco":
        scheme, kw = "det", dict(kw, det_dataflow=2)
    return db.run(scheme, batch, eng.params(**kw) if kw else None, timeout_s=timeout_s)


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine
    return engine


def check(table, final, batch, res, reads, scheme, stats=None, require_all=True):
    rep = oracle.replay_check(table, final, batch, res, reads, require_all=require_all)
    assert rep["ok"], (scheme, rep, stats)
    if scheme.startswith("det"):
        ref_final, ref_reads = oracle.serial(table, batch)
        committed = res["status"] == oracle.ST_COMMITTED
        assert committed.all()
        assert np.array_equal(res["commit_order"], np.arange(batch.n_txns))
        assert np.array_equal(final, ref_final) and np.array_equal(reads, ref_reads)
    return rep


@pytest.mark.parametrize("scheme", SCHEMES)
def test_small_kv_store(eng, scheme):
    """65,536 records x 8 u64 fields, 4,096 txns x 16 uniform keys, one launch."""
    table, batch = wl.small_kv()
    with eng.Database("kv", n_records=65536, n_fields=8, field_bytes=8,
                      max_batch_txns=4096) as db:
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, batch)
        final = db.read_kv()
    assert stats["committed"] == 4096 and stats["device_error"] == 0, stats
    check(table, final, batch, res, reads, scheme, stats)
    # every op's read value appears in the output, rmw results applied
    assert not np.array_equal(final, table)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 32])
def test_lane_group_widths(eng, scheme, lanes):
    """Hot keys, ragged op counts (1..40 ops, several per lane) for every lane-group width."""
    nrec = 16384
    table = wl.kv_table_splitmix(77, nrec, 4)
    batch = wl.kv_batch(5 + lanes, nrec=nrec, nfields=4, n_txns=3000, ops_range=(1, 40),
                        read_ratio=0.5, theta=0.6)
    with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8, max_ops_per_txn=40,
                      max_batch_txns=3000) as db:
        db.load_kv(table)
        # 1 lane per txn stages 32 txns x 40 ops per warp: keep the block small
        res, reads, stats = go(eng, db, scheme, batch, lanes_per_txn=lanes,
                               warps_per_block=2 if lanes == 1 else 4, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, scheme, stats)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_sixteen_byte_slots_contention(eng, scheme):
    """16-byte slots (10 payload bytes), Zipf 0.99, 2^15 txns, several tiles."""
    nrec, nf = 1 << 16, 10
    table = wl.kv_table_bytes(3, nrec, nf)
    batch = wl.kv_batch(4, nrec=nrec, nfields=nf, n_txns=1 << 15, read_ratio=0.5, theta=0.9,
                        field_bytes=16)
    with eng.Database("kv", n_records=nrec, n_fields=nf, field_bytes=16,
                      max_batch_txns=1 << 15) as db:
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, batch, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, scheme, stats)
    raw = final.view(np.uint8).reshape(nf, nrec, 16)
    assert not raw[..., 10:].any()          # padding bytes stay zero


@pytest.mark.parametrize("scheme", SCHEMES)
def test_tiny_batches_brute_force(eng, scheme):
    """Batches of <= 6 txns on 3 hot records: the outcome equals at least one
    serial order (brute force), and the replay in the reported order."""
    rng = np.random.default_rng(17)
    with eng.Database("kv", n_records=8, n_fields=1, field_bytes=8, max_ops_per_txn=3,
                      max_batch_txns=8) as db:
        for trial in range(12):
            n = int(rng.integers(2, 7))
            lists = []
            for _ in range(n):
                ks = rng.permutation(3)[: int(rng.integers(1, 4))]
                lists.append([(int(k), 0, int(rng.integers(0, 2)), int(rng.integers(1, 99)), 0)
                              for k in ks])
            batch = wl.kv_batch_from_lists(lists)
            table = rng.integers(0, 1000, size=(1, 8), dtype=np.uint64)
            db.load_kv(table)
            res, reads, stats = go(eng, db, scheme, batch, lanes_per_txn=1)
            final = db.read_kv()
            m, _ = oracle.brute_force(table, batch, final, reads)
            assert m >= 1, (scheme, trial)
            check(table, final, batch, res, reads, scheme, stats)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_edge_cases(eng, scheme):
    with eng.Database("kv", n_records=64, n_fields=2, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=16) as db:
        table = wl.kv_table_splitmix(1, 64, 2)
        db.load_kv(table)
        # empty batch
        empty = wl.kv_batch_from_lists([])
        res, reads, stats = go(eng, db, scheme, empty)
        assert stats["committed"] == 0 and res.size == 0
        # read-only batch: reads are the initial values, table unchanged
        ro = wl.kv_batch(2, nrec=64, nfields=2, n_txns=16, ops_per_txn=4, read_ratio=1.0)
        res, reads, stats = go(eng, db, scheme, ro)
        assert np.array_equal(db.read_kv(), table)
        assert np.array_equal(reads[:, 0], table[ro.ops["field"], ro.ops["key"]])
        # malformed transactions come back INVALID, the others commit
        bad = wl.kv_batch_from_lists([
            [(3, 0, 1, 5, 0), (3, 1, 0, 0, 0)],     # duplicate key
            [(64, 0, 0, 0, 0)],                     # key out of range
            [(1, 2, 0, 0, 0)],                      # field out of range
            [(2, 0, 9, 0, 0)],                      # unknown kind
            [(5, 1, 1, 7, 0)],                      # fine
        ])
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, bad)
        assert res["status"].tolist() == [3, 3, 3, 3, 1]
        assert stats["invalid"] == 4 and "invalid" in stats["errors"]
        final = db.read_kv()
        assert int(final[1, 5]) == (int(table[1, 5]) + 7) % (1 << 64)
        assert int(reads[5, 0]) == int(table[1, 5])          # op 5: the valid txn's op
        # an out-of-range key between two valid writers of record 0: with a
        # power-of-two record count the marker key of out-of-range accesses
        # (64) must still sort after record 0's accesses, so that the two
        # writers run in id order and nothing waits on the marker
        mixed = wl.kv_batch_from_lists([
            [(0, 0, 1, 5, 0), (9, 1, 0, 0, 0)],
            [(64, 0, 1, 0, 0), (0, 1, 1, 3, 0)],     # key out of range
            [(0, 0, 1, 7, 0)],
            [(9, 1, 1, 11, 0), (0, 1, 0, 0, 0)],
        ])
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, mixed, wait_budget_ns=200_000_000)
        assert res["status"].tolist() == [1, 3, 1, 1], (res, stats)
        assert stats["timeouts"] == 0
        final = db.read_kv()
        rep = oracle.replay_check(table, final, mixed, res, reads, require_all=False)
        assert rep["ok"] and rep["n_committed"] == 3, rep
        if scheme.startswith("det"):
            valid = [0, 2, 3]
            ref_final, ref_reads = oracle.serial(table, mixed, order=valid)
            assert np.array_equal(final, ref_final)
            ops = np.concatenate([np.arange(f, f + n) for f, n in
                                  zip(mixed.txns["first_op"][valid], mixed.txns["n_ops"][valid])])
            assert np.array_equal(reads[ops], ref_reads[ops])
            assert res["commit_order"][valid].tolist() == [0, 1, 2]
        # capacity is enforced on the host
        big = wl.kv_batch(3, nrec=64, nfields=2, n_txns=17, ops_per_txn=2)
        with pytest.raises(eng.GCCError):
            db.submit("det" if scheme.startswith("det") else scheme, big)


@pytest.mark.parametrize("field_bytes", [8, 16])
def test_seeded_init_on_the_device(eng, field_bytes):
    """gcc_init_table_seeded writes the generator's table bit for bit and
    resets the control words: a batch afterwards replays from that table."""
    nrec, nfields = 3001, 3                         # slots not a multiple of the block
    table = wl.kv_table_seeded(0x5EED0009, nrec, nfields, field_bytes)
    with eng.Database("kv", n_records=nrec, n_fields=nfields, field_bytes=field_bytes,
                      max_batch_txns=2048) as db:
        db.init_seeded(0x5EED0009)
        assert np.array_equal(db.read_kv(), table)
        batch = wl.kv_batch(12, nrec=nrec, nfields=nfields, n_txns=2048, theta=0.8,
                            field_bytes=field_bytes)
        res, reads, stats = go(eng, db, "occ", batch)
        check(table, db.read_kv(), batch, res, reads, "occ", stats)
        db.init_seeded(0x5EED0009)                    # again, after the batch
        assert np.array_equal(db.read_kv(), table)


def test_outstanding_batch_limit(eng):
    """Up to GCC_MAX_OUTSTANDING_BATCHES (256) submitted batches may be pending
    on one database; one more is refused with GCC_ERR_CAPACITY until a batch
    is freed.  Waited in reverse order, every batch still returns its own
    reads and statistics: deterministic batches equal serial execution of the
    batches in submission order, transaction by transaction."""
    nrec = 256
    state = wl.kv_table_splitmix(11, nrec, 2)
    with eng.Database("kv", n_records=nrec, n_fields=2, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=16) as db:
        db.load_kv(state)
        batches = [wl.kv_batch(1000 + i, nrec=nrec, nfields=2, n_txns=16, ops_per_txn=4,
                               theta=0.8) for i in range(258)]
        handles = [db.submit("det", b) for b in batches[:256]]
        with pytest.raises(eng.GCCError) as err:
            db.submit("det", batches[256])
        assert err.value.status == 6
        expect = []
        for b in batches[:256]:
            state, reads = oracle.serial(state, b)
            expect.append(reads)
        # the oldest batch is released unread; its slot takes the next batch
        handles[0].free()
        handles[0] = db.submit("det", batches[256])
        state, reads = oracle.serial(state, batches[256])
        expect[0] = reads
        for i in reversed(range(256)):
            res, got, stats = handles[i].wait(120)
            handles[i].free()
            assert stats["committed"] == 16 and stats["device_error"] == 0, (i, stats)
            assert np.array_equal(got, expect[i]), i
        assert np.array_equal(db.read_kv(), state)


@pytest.mark.parametrize("scheme", ["occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc"])
def test_injected_aborts_and_backoff(eng, scheme):
    """Forced aborts at the commit point (30%) and randomized backoff exercise
    the retry path; the outcome still replays exactly."""
    table, batch = wl.small_kv(seed=9, n_txns=2048, nrec=4096)
    with eng.Database("kv", n_records=4096, n_fields=8, field_bytes=8,
                      max_batch_txns=2048) as db:
        db.load_kv(table)
        p = eng.params(inject_abort_ppm=300000, backoff_base_ns=200, backoff_cap_ns=20000,
                       seed=1234)
        res, reads, stats = db.run(scheme, batch, p)
        final = db.read_kv()
    assert stats["aborts"] > 0.2 * batch.n_txns, stats
    assert (res["attempts"] > 1).any()
    check(table, final, batch, res, reads, scheme, stats)


def test_attempt_budget_gives_up_cleanly(eng):
    """With every attempt forced to abort and a budget of 3 attempts, each txn
    ends TIMEOUT after exactly 3 attempts, no lock is left behind, and the next
    batch on the same database runs normally."""
    table, batch = wl.small_kv(seed=2, n_txns=256, nrec=1024)
    with eng.Database("kv", n_records=1024, n_fields=8, field_bytes=8,
                      max_batch_txns=256) as db:
        db.load_kv(table)
        for scheme in ("2pl", "2pl_wd", "occ", "to", "tictoc", "mvcc"):
            res, reads, stats = db.run(scheme, batch,
                                       eng.params(inject_abort_ppm=1000000, max_attempts=3))
            assert (res["status"] == oracle.ST_TIMEOUT).all(), scheme
            assert (res["attempts"] == 3).all()
            assert "attempts" in stats["errors"]
            assert np.array_equal(db.read_kv(), table)
        res, reads, stats = db.run("2pl", batch)
        check(table, db.read_kv(), batch, res, reads, "2pl", stats)


@pytest.mark.parametrize("scheme", ["occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc"])
@pytest.mark.parametrize("policy", [dict(retry_queue=2), dict(queue_after=1),
                                    dict(queue_after=1, queue_width=4),
                                    dict(queue_after=3, queue_turn_ns=200)],
                         ids=["off", "first-abort", "width4", "after3"])
def test_retry_policies_replay(eng, scheme, policy):
    """Zipf 0.99 over 4,096 records: with retry queues off, joined from the
    first abort, admitting four at once, or joined after three aborts, every
    txn commits and the history replays exactly."""
    nrec = 1 << 12
    table = wl.kv_table_splitmix(21, nrec, 2)
    batch = wl.kv_batch(22, nrec=nrec, nfields=2, n_txns=4096, read_ratio=0.5, theta=0.99)
    with eng.Database("kv", n_records=nrec, n_fields=2, field_bytes=8, max_batch_txns=4096) as db:
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, batch, **HOT, **policy)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, scheme, stats)


@pytest.mark.parametrize("scheme", ["occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc"])
def test_retry_queues_after_a_deadline(eng, scheme):
    """A hot batch cut off by a 1 ms kernel deadline while transactions wait in
    retry queues ends with TIMEOUT statuses and the deadline flag; what did
    commit replays exactly, and the next batch on the database starts from
    clean queues and commits everything."""
    nrec = 1 << 10
    table = wl.kv_table_splitmix(23, nrec, 2)
    batch = wl.kv_batch(24, nrec=nrec, nfields=2, n_txns=16384, read_ratio=0.5, theta=0.99)
    with eng.Database("kv", n_records=nrec, n_fields=2, field_bytes=8, max_batch_txns=16384) as db:
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, batch, deadline_ns=1_000_000, queue_after=1)
        state = db.read_kv()
        if stats["timeouts"]:
            assert "deadline" in stats["errors"], stats
            assert (res["status"] == oracle.ST_TIMEOUT).sum() == stats["timeouts"]
        assert stats["committed"] + stats["timeouts"] == batch.n_txns, stats
        check(table, state, batch, res, reads, scheme, stats, require_all=False)
        res, reads, stats = go(eng, db, scheme, batch, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(state, final, batch, res, reads, scheme, stats)


def test_det_wait_budget_returns(eng):
    """A deterministic-scheme wait that runs out of budget ends the batch with
    TIMEOUT statuses and an error flag instead of hanging; the database is
    usable afterwards."""
    nrec = 64
    table = wl.kv_table_splitmix(4, nrec, 1)
    # one very hot record: long chains of dependent writes
    batch = wl.kv_batch(6, nrec=nrec, nfields=1, n_txns=20000, ops_per_txn=4, theta=0.99,
                        read_ratio=0.0)
    with eng.Database("kv", n_records=nrec, n_fields=1, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=20000) as db:
        db.load_kv(table)
        res, reads, stats = db.run("det", batch, eng.params(wait_budget_ns=1000, det_dataflow=1))
        if stats["device_error"]:
            assert "wait_budget" in stats["errors"]
            assert (res["status"] == oracle.ST_TIMEOUT).any()
        db.load_kv(table)
        res, reads, stats = db.run("det", batch, eng.params(det_dataflow=1))
        check(table, db.read_kv(), batch, res, reads, "det", stats)


def test_det_gap_in_op_ranges_runs_out_its_waits(eng):
    """A deterministic batch whose transaction op ranges leave an op out: run
    op by op, a later access to that op's record waits for it, the wait runs
    out of its (short) budget, and the transaction ends TIMEOUT with the
    wait-budget flag while the others commit; the prefix-sum path leaves the
    uncovered op out of its access table and commits everything.  The
    database is usable afterwards."""
    nrec = 16
    table = wl.kv_table_splitmix(5, nrec, 1)
    full = wl.kv_batch_from_lists([
        [(1, 0, 1, 5, 0), (2, 0, 0, 0, 0)],
        [(7, 0, 1, 9, 0)],                              # becomes the uncovered op
        [(7, 0, 1, 3, 0), (3, 0, 0, 0, 0)],
    ])
    txns = full.txns[[0, 2]].copy()                     # op 2 belongs to no transaction
    gap = wl.KVBatch(txns=txns, ops=full.ops, operands=full.operands)
    with eng.Database("kv", n_records=nrec, n_fields=1, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=8) as db:
        db.load_kv(table)
        res, reads, stats = db.run("det", gap, eng.params(det_dataflow=1,
                                                         wait_budget_ns=20_000_000))
        assert res["status"].tolist() == [oracle.ST_COMMITTED, oracle.ST_TIMEOUT], res
        assert "wait_budget" in stats["errors"]
        db.load_kv(table)
        res, reads, stats = db.run("det", gap)
        assert (res["status"] == oracle.ST_COMMITTED).all()
        ref = oracle.serial(table, wl.KVBatch(txns=txns, ops=full.ops, operands=full.operands))
        assert np.array_equal(db.read_kv(), ref[0])


def test_schemes_share_one_database(eng):
    """Schemes alternate on one database; each batch starts from the previous
    batch's final state and replays exactly."""
    nrec = 1 << 14
    state = wl.kv_table_splitmix(8, nrec, 4)
    with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8,
                      max_batch_txns=4096) as db:
        db.load_kv(state)
        for i, scheme in enumerate(["occ", "occ", "2pl", "det", "to", "occ", "det-dataflow",
                                    "tictoc", "tictoc", "2pl", "2pl_wd", "to", "tictoc",
                                    "2pl_wd", "det", "mvcc", "mvcc", "occ", "mvcc", "to",
                                    "mvcc", "det", "mvcc", "2pl"]):
            batch = wl.kv_batch(100 + i, nrec=nrec, nfields=4, n_txns=4096, theta=0.8)
            res, reads, stats = go(eng, db, scheme, batch)
            final = db.read_kv()
            check(state, final, batch, res, reads, scheme, stats)
            state = final


@pytest.mark.slow
@pytest.mark.parametrize("theta,read_ratio", [(0.0, 0.5), (0.6, 0.5), (0.8, 0.5), (0.99, 0.5),
                                              (0.6, 0.95), (0.8, 0.95), (0.99, 0.95)])
def test_ycsb_full_size(eng, theta, read_ratio):
    """2^24 records x 10 fields in 16-byte slots, 2^20 txns x 16 ops, at the
    contention levels of the key-value sweep (Zipf 0, 0.6, 0.8, 0.99 at read
    ratio 0.5; 0.6, 0.8, 0.99 at 0.95): every scheme in turn on one database,
    each batch replayed in full by the oracle (the launch shape is the
    benchmark's)."""
    table, batch = wl.ycsb_kv(theta=theta, read_ratio=read_ratio)
    state = table
    with eng.Database("kv", n_records=1 << 24, n_fields=10, field_bytes=16,
                      max_batch_txns=1 << 20) as db:
        db.load_kv(state)
        for scheme in SCHEMES:
            res, reads, stats = go(eng, db, scheme, batch, timeout_s=300)
            final = db.read_kv()
            assert stats["committed"] == batch.n_txns, (scheme, stats)
            rep = oracle.replay_check(state, final, batch, res, reads)
            assert rep["ok"], (scheme, rep)
            state = final


def test_tictoc_hot_reads_replay(eng):
    """TicToc skips re-checking a read whose read timestamp already covers the
    commit timestamp, so every read must be a consistent (wts, value, rts)
    snapshot: read-mostly batches on a few very hot records, several in a row,
    replay exactly."""
    nrec = 1 << 10
    state = wl.kv_table_splitmix(31, nrec, 2)
    with eng.Database("kv", n_records=nrec, n_fields=2, field_bytes=8, max_batch_txns=16384) as db:
        db.load_kv(state)
        for i in range(4):
            batch = wl.kv_batch(32 + i, nrec=nrec, nfields=2, n_txns=16384, read_ratio=0.9,
                                theta=0.99)
            res, reads, stats = go(eng, db, "tictoc", batch, **HOT)
            final = db.read_kv()
            assert stats["committed"] == batch.n_txns, stats
            check(state, final, batch, res, reads, "tictoc", stats)
            state = final


@pytest.mark.parametrize("scheme", SCHEMES)
def test_hot_key_zipf_099(eng, scheme):
    """Zipf 0.99 over 2^16 records, 4,096 txns x 16 ops: the hottest record is
    in several percent of all ops; every scheme still commits everything and
    replays exactly."""
    nrec = 1 << 16
    table = wl.kv_table_splitmix(12, nrec, 2)
    batch = wl.kv_batch(13, nrec=nrec, nfields=2, n_txns=4096, read_ratio=0.5, theta=0.99)
    with eng.Database("kv", n_records=nrec, n_fields=2, field_bytes=8, max_batch_txns=4096) as db:
        db.load_kv(table)
        res, reads, stats = go(eng, db, scheme, batch, **HOT)
        final = db.read_kv()
    assert stats["committed"] == batch.n_txns, stats
    check(table, final, batch, res, reads, scheme, stats)

