"""GPU parity of the served form (continuous batching over a request trace).

A lane's committed requests, ordered by (batch_seq, commit_order), are one
serial history of its database: the oracle replays that history from the
initial state and must reproduce every read and the final state.  Requests on
disjoint keys get bit-identical results alone and mixed with other traffic.
"""
import numpy as np
import pytest

import oracle
from paper_2406_10158_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine
    return engine


def lane_history(trace, lane_of, comp, reads, lane):
    """(sub-batch in serial order, results with dense commit ranks, reads)."""
    idx = np.nonzero(lane_of == lane)[0]
    c = comp[idx]
    assert (c["status"] == oracle.ST_COMMITTED).all()
    order = np.lexsort((c["commit_order"], c["batch_seq"]))
    sub = wl.select(trace, idx)
    res = np.zeros(idx.size, dtype=wl.RESULT_DTYPE)
    res["status"] = oracle.ST_COMMITTED
    res["commit_order"][order] = np.arange(idx.size)
    first = trace.txns["first_op"][idx].astype(np.int64)
    nops = trace.txns["n_ops"][idx].astype(np.int64)
    src = np.repeat(first, nops) + (np.arange(int(nops.sum())) -
                                    np.repeat(np.concatenate([[0], np.cumsum(nops)[:-1]]), nops))
    return sub, res, reads[src]


@pytest.mark.parametrize("schemes", [("occ", "occ"), ("det", "2pl"), ("to", "det")])
def test_served_mix_replays(eng, schemes):
    nrec, W = 1 << 14, 2
    table = wl.kv_table_splitmix(21, nrec, 8)
    kv = wl.kv_batch(22, nrec=nrec, nfields=8, n_txns=4000, read_ratio=0.8, theta=0.8)
    oe0, oe, cap = wl.order_entry(seed=23, W=W, n_txns=4000)
    rng = np.random.default_rng(1)
    lane_of = (rng.random(6000) < 0.5).astype(np.uint32)          # 0 = KV, 1 = order entry
    trace = wl.interleave([kv, oe], lane_of)
    arrivals = wl.poisson_arrivals(24, 6000, 2e6)
    with eng.Database("kv", n_records=nrec, n_fields=8, field_bytes=8, max_batch_txns=512) as dkv, \
            eng.Database("oe", n_warehouses=W, order_cap=cap, max_ops_per_txn=33,
                         max_batch_txns=512, max_batch_ops=512 * 33) as doe:
        dkv.load_kv(table)
        doe.load_oe(oe0)
        srv = eng.Server([(dkv, schemes[0], 512, 0, 50_000, 3), (doe, schemes[1], 512, 0, 50_000, 3)],
                         eng.params(backoff_cap_ns=16_000_000))
        comp, reads = srv.run_trace(lane_of, trace, arrivals)
        tot = [srv.lane_totals(0), srv.lane_totals(1)]
        srv.close()
        final_kv, final_oe = dkv.read_kv(), doe.read_oe()
    assert tot[0]["batches"] > 1 and tot[1]["batches"] > 1
    assert (comp["done_ns"] >= comp["arrival_ns"]).all()
    sub, res, rd = lane_history(trace, lane_of, comp, reads, 0)
    rep = oracle.replay_check(table, final_kv, sub, res, rd)
    assert rep["ok"], rep
    sub, res, rd = lane_history(trace, lane_of, comp, reads, 1)
    rep = oracle.oe_replay_check(oe0, final_oe, W, cap, sub, res, rd)
    assert rep["ok"], rep
    assert oracle.oe_consistency(final_oe, W, cap) == 0


@pytest.mark.slow
def test_served_full_size_replays(eng):
    """The served workload at full size: 2^24 records x 8 u64 fields (Zipf
    0.8, 80% reads) under OCC on one lane and order entry at W = 8 under
    basic TO on the other, 2^17 requests 50/50 at 10^7 txn/s offered, the
    benchmark's batch cap, delay and depth; both lanes' histories replay
    exactly and the order-entry database stays consistent."""
    nrec, W, n = 1 << 24, 8, 1 << 17
    table = wl.kv_table_splitmix(wl.SEEDS[4], nrec, 8)
    kv = wl.kv_batch(wl.derive_seed(wl.SEEDS[4], 1), nrec=nrec, nfields=8, n_txns=n,
                     read_ratio=0.8, theta=0.8)
    oe0, oe, cap = wl.order_entry(seed=wl.SEEDS[4], W=W, n_txns=n)
    rng = np.random.default_rng(7)
    lane_of = (rng.random(n) < 0.5).astype(np.uint32)
    trace = wl.interleave([kv, oe], lane_of)
    arrivals = wl.poisson_arrivals(wl.SEEDS[4] + 7, n, 1e7)
    mb = 1 << 14
    with eng.Database("kv", n_records=nrec, n_fields=8, field_bytes=8, max_batch_txns=mb) as dkv, \
            eng.Database("oe", n_warehouses=W, order_cap=cap, max_ops_per_txn=33,
                         max_batch_txns=mb, max_batch_ops=mb * 33) as doe:
        dkv.load_kv(table)
        doe.load_oe(oe0)
        srv = eng.Server([(dkv, "occ", mb, 0, 100_000, 4), (doe, "to", mb, 0, 100_000, 4)],
                         eng.params(backoff_cap_ns=16_000_000))
        comp, reads = srv.run_trace(lane_of, trace, arrivals)
        srv.close()
        final_kv, final_oe = dkv.read_kv(), doe.read_oe()
    assert (comp["status"] == oracle.ST_COMMITTED).all()
    sub, res, rd = lane_history(trace, lane_of, comp, reads, 0)
    rep = oracle.replay_check(table, final_kv, sub, res, rd)
    assert rep["ok"], rep
    sub, res, rd = lane_history(trace, lane_of, comp, reads, 1)
    rep = oracle.oe_replay_check(oe0, final_oe, W, cap, sub, res, rd)
    assert rep["ok"], rep
    assert oracle.oe_consistency(final_oe, W, cap) == 0


@pytest.mark.parametrize("scheme", ["occ", "det"])
def test_served_same_alone_and_in_the_mix(eng, scheme):
    """Requests on disjoint keys: identical reads and final table whether they
    are served alone or interleaved with order-entry traffic (tolerance 0)."""
    nrec, W = 1 << 16, 1
    table = wl.kv_table_splitmix(31, nrec, 4)
    kv = wl.disjoint_kv(32, 2000, nrec, 4)
    oe0, oe, cap = wl.order_entry(seed=33, W=W, n_txns=3000)
    outcomes = []
    for mixed in (False, True):
        if mixed:
            lane_of = np.zeros(5000, dtype=np.uint32)
            lane_of[np.random.default_rng(2).permutation(5000)[:3000]] = 1
        else:
            lane_of = np.zeros(2000, dtype=np.uint32)
        trace = wl.interleave([kv, oe], lane_of)
        arrivals = wl.poisson_arrivals(34, lane_of.size, 1e6)
        with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8, max_batch_txns=256) as dkv, \
                eng.Database("oe", n_warehouses=W, order_cap=cap, max_ops_per_txn=33,
                             max_batch_txns=256, max_batch_ops=256 * 33) as doe:
            dkv.load_kv(table)
            doe.load_oe(oe0)
            srv = eng.Server([(dkv, scheme, 256, 0, 30_000, 2), (doe, "occ", 256, 0, 30_000, 2)])
            comp, reads = srv.run_trace(lane_of, trace, arrivals)
            srv.close()
            final = dkv.read_kv()
        kv_idx = np.nonzero(lane_of == 0)[0]
        assert (comp["status"][kv_idx] == oracle.ST_COMMITTED).all()
        sub = wl.select(trace, kv_idx)
        first = trace.txns["first_op"][kv_idx].astype(np.int64)
        kv_reads = np.concatenate([reads[f:f + 16] for f in first])
        outcomes.append((kv_reads, final, sub))
    (r0, f0, s0), (r1, f1, s1) = outcomes
    assert np.array_equal(s0.ops, s1.ops)
    assert np.array_equal(r0, r1)
    assert np.array_equal(f0, f1)
    # and both equal the serial execution of the requests
    ref_final, ref_reads = oracle.serial(table, s0)
    assert np.array_equal(ref_final, f0) and np.array_equal(ref_reads, r0)


def test_server_drains_after_the_producer_stops(eng):
    """A producer enqueues requests in bursts, pumping between them, and then
    stops mid-stream: drain completes every admitted request, and their
    history replays exactly."""
    nrec = 1 << 12
    table = wl.kv_table_splitmix(51, nrec, 4)
    kv = wl.kv_batch(52, nrec=nrec, nfields=4, n_txns=3000, read_ratio=0.5, theta=0.9)
    with eng.Database("kv", n_records=nrec, n_fields=4, field_bytes=8, max_batch_txns=256) as db:
        db.load_kv(table)
        srv = eng.Server([(db, "occ", 256, 0, 50_000, 3)], eng.params(backoff_cap_ns=16_000_000))
        try:
            sent = 0
            for burst in range(7):                      # then the producer stops
                for t in range(sent, sent + 300):
                    f, nops = int(kv.txns["first_op"][t]), int(kv.txns["n_ops"][t])
                    srv.enqueue(0, kv.txns[t:t + 1], kv.ops[f:f + nops],
                                kv.operands[f:f + nops].astype(np.uint64), srv.now_ns())
                sent += 300
                srv.pump()
            srv.drain()
            comp, reads = srv.completions()
        finally:
            srv.close()
        final = db.read_kv()
    assert comp.size == sent and (comp["status"] == oracle.ST_COMMITTED).all()
    sub = wl.select(kv, comp["request"].astype(np.int64))
    res = np.zeros(comp.size, dtype=wl.RESULT_DTYPE)
    res["status"] = oracle.ST_COMMITTED
    order = np.lexsort((comp["commit_order"], comp["batch_seq"]))
    res["commit_order"][order] = np.arange(comp.size)
    assert np.array_equal(np.sort(comp["request"]), np.arange(sent))
    rep = oracle.replay_check(table, final, sub, res, reads[:sub.n_ops])
    assert rep["ok"], rep


def test_server_rejects_requests_larger_than_a_batch(eng):
    """A database whose batches hold fewer ops than a transaction may have:
    a request that no batch of its lane can hold is refused on the host
    (enqueue: capacity; trace: invalid, nothing run); one that fits is served."""
    table = wl.kv_table_splitmix(41, 64, 2)
    big = wl.kv_batch_from_lists([[(1, 0, 1, 5, 0), (2, 0, 0, 0, 0), (3, 1, 1, 9, 0)]])
    small = wl.kv_batch_from_lists([[(4, 0, 1, 7, 0), (5, 1, 0, 0, 0)]])
    with eng.Database("kv", n_records=64, n_fields=2, field_bytes=8, max_ops_per_txn=4,
                      max_batch_txns=8, max_batch_ops=2) as db:
        db.load_kv(table)
        srv = eng.Server([(db, "occ", 8, 0, 30_000, 2)])
        try:
            with pytest.raises(eng.GCCError) as err:
                srv.enqueue(0, big.txns[:1], big.ops, big.operands.astype(np.uint64),
                            srv.now_ns())
            assert err.value.status == 6
            with pytest.raises(eng.GCCError) as err:
                srv.run_trace(np.zeros(1, dtype=np.uint32), big, np.zeros(1, dtype=np.uint64))
            assert err.value.status == 1
            srv.enqueue(0, small.txns[:1], small.ops, small.operands.astype(np.uint64),
                        srv.now_ns())
            srv.drain()
            comp, reads = srv.completions()
        finally:
            srv.close()
        final = db.read_kv()
    assert comp.size == 1 and comp["status"][0] == oracle.ST_COMMITTED
    assert int(reads[0, 0]) == int(table[0, 4]) and int(reads[1, 0]) == int(table[1, 5])
    assert int(final[0, 4]) == (int(table[0, 4]) + 7) % (1 << 64)
    assert np.array_equal(np.delete(final.ravel(), 4), np.delete(table.ravel(), 4))
