"""The seeded input generators (CPU only): shapes, ranges and distributions."""
import numpy as np

from paper_2406_10158_gb300 import workload as wl


def test_feistel_is_a_bijection():
    for n in (1 << 10, 1000, 65536):
        p = wl.feistel_permute(np.arange(n, dtype=np.uint64), n, 7)
        assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint64))


def test_keys_distinct_within_each_transaction():
    b = wl.kv_batch(3, nrec=64, nfields=2, n_txns=500, ops_per_txn=16, theta=0.99)
    k = b.ops["key"].reshape(500, 16)
    s = np.sort(k, axis=1)
    assert not (s[:, 1:] == s[:, :-1]).any()
    assert (k < 64).all()


def test_zipf_head_frequency_matches_closed_form():
    """Rank 0 of Zipf(theta) over N items has probability 1 / zeta(N, theta)."""
    rng = np.random.default_rng(0)
    n, theta, draws = 1 << 16, 0.8, 400_000
    r = wl.zipf_ranks(rng, n, theta, draws)
    zeta = np.sum(np.arange(1, n + 1, dtype=np.float64) ** -theta)
    p0 = 1.0 / zeta
    got = np.count_nonzero(r == 0) / draws
    assert abs(got - p0) < 5 * np.sqrt(p0 / draws)
    assert r.max() < n
    u = wl.zipf_ranks(rng, n, 0.0, draws)           # theta 0 = uniform
    assert abs(np.mean(u) / (n - 1) - 0.5) < 0.01


def test_nurand_range_and_read_ratio():
    rng = np.random.default_rng(1)
    x = wl.nurand(rng, 8191, 1, 100000, 123, 100000)
    assert x.min() >= 1 and x.max() <= 100000
    b = wl.kv_batch(4, nrec=4096, nfields=8, n_txns=4000, read_ratio=0.8)
    frac = np.mean(b.ops["kind"] == wl.OP_READ)
    assert abs(frac - 0.8) < 0.01
    assert not b.operands[b.ops["kind"] == wl.OP_READ].any()


def test_hotspot_batch_shape():
    _, b = wl.kv_hotspot(3, hot_frac=0.1, nrec=1 << 16, n_txns=4096, with_table=False)
    keys = b.ops["key"].reshape(-1, 16)
    assert all(len(set(r)) == 16 for r in keys)
    hot = (keys == 12345)
    writes = hot & (b.ops["kind"].reshape(-1, 16) == wl.OP_ADD)
    share = hot.any(axis=1).mean()
    assert 0.08 < share < 0.12
    # the hot record is written by (nearly) every transaction that touches it
    assert writes.sum() >= 0.95 * hot.sum()


def test_order_entry_shapes():
    db, b, cap = wl.order_entry(seed=5, W=2, n_txns=2000)
    t = b.txns
    no = t["type"] == wl.TXN_NEW_ORDER
    assert ((t["n_ops"][no] >= 5) & (t["n_ops"][no] <= 33)).all()
    assert (t["n_ops"][~no] == 3).all()
    assert abs(no.mean() - 0.5) < 0.05
    assert cap >= 3000


def test_trace_interleave_and_select_round_trip():
    kv = wl.kv_batch(1, nrec=1000, nfields=2, n_txns=50, ops_per_txn=3)
    _, oe, _ = wl.order_entry(seed=2, W=1, n_txns=40)
    lane_of = np.array([0] * 30 + [1] * 40 + [0] * 20, dtype=np.uint32)
    np.random.default_rng(0).shuffle(lane_of)
    tr = wl.interleave([kv, oe], lane_of)
    assert tr.n_txns == 90
    s0 = wl.select(tr, np.nonzero(lane_of == 0)[0])
    s1 = wl.select(tr, np.nonzero(lane_of == 1)[0])
    k, o = wl.select(kv, np.arange(50)), wl.select(oe, np.arange(40))
    assert np.array_equal(s0.ops, k.ops) and np.array_equal(s0.operands, k.operands)
    assert np.array_equal(s1.ops, o.ops) and np.array_equal(s1.txns, o.txns)
    a = wl.poisson_arrivals(3, 10000, 1e6)
    assert (np.diff(a.astype(np.int64)) >= 0).all()
    assert abs(float(a[-1]) / 1e4 - 1000.0) < 50.0          # mean gap 1 us


def test_batched_databases_in_range():
    """64 databases: 2^16..2^22 records, 1,000..262,144 txns of 4..64 ops
    (sizes drawn log-uniformly); here with small bounds to stay fast."""
    spec = wl.batched_kv(9, n_db=6, rec_bits=(10, 12), txn_range=(100, 400), ops_range=(4, 64))
    assert len(spec) == 6
    for nrec, table, batch in spec:
        assert nrec in (1 << 10, 1 << 11, 1 << 12)
        assert table.shape == (8, nrec)
        assert 100 <= batch.n_txns <= 400
        n = batch.txns["n_ops"]
        assert n.min() >= 4 and n.max() <= 64
        assert (batch.ops["key"] < nrec).all()
        # op ranges tile the op array in transaction-id order
        first = batch.txns["first_op"].astype(np.int64)
        assert first[0] == 0 and np.array_equal(first[1:], np.cumsum(n.astype(np.int64))[:-1])


def test_poisson_arrivals_have_the_offered_rate():
    rate, n = 1e6, 200_000
    t = wl.poisson_arrivals(3, n, rate).astype(np.float64)
    gaps = np.diff(t)
    assert (gaps >= 0).all()
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() / (1e9 / rate) - 1.0) < 0.01
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02


def test_customer_names():
    names = wl.oe_customer_names(3, 2)
    last = names["c_last"].reshape(2 * wl.OE_DISTRICTS, wl.OE_CUSTOMERS)
    assert names["c_first"].shape == last.ravel().shape
    assert (last[:, :wl.OE_LAST_NAMES] == np.arange(wl.OE_LAST_NAMES)).all()
    assert last.min() >= 0 and last.max() < wl.OE_LAST_NAMES
    # NURand skews the remaining 2,000 per district towards a few names
    counts = np.bincount(last[:, wl.OE_LAST_NAMES:].ravel(), minlength=wl.OE_LAST_NAMES)
    assert counts.max() > 4 * counts.mean()


def test_payments_by_last_name_share_and_encoding():
    """by_name_frac = 0 leaves every payment by id (the same batch as without
    the option); 0.6 names about 60% of the customers by last name, keyed by
    the customer's district with a last-name id that exists there."""
    _, b0, _ = wl.order_entry(seed=9, W=2, n_txns=4000)
    _, b1, _ = wl.order_entry(seed=9, W=2, n_txns=4000, by_name_frac=0.6)
    assert not (b0.ops["kind"] == wl.OE_C_PAY_BY_NAME).any()
    pay = b1.txns["type"] == wl.TXN_PAYMENT
    third = b1.txns["first_op"][pay].astype(np.int64) + 2
    by_name = b1.ops["kind"][third] == wl.OE_C_PAY_BY_NAME
    assert 0.55 < by_name.mean() < 0.65
    assert (b1.ops["key"][third[by_name]] < 2 * wl.OE_DISTRICTS).all()
    assert (b1.ops["aux"][third[by_name]] < wl.OE_LAST_NAMES).all()
    same = np.ones(b1.n_ops, dtype=bool)
    same[third[by_name]] = False
    assert np.array_equal(b0.ops[same], b1.ops[same])
    assert np.array_equal(b0.operands, b1.operands)
