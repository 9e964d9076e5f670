"""GPU parity of the order-entry path (NewOrder / Payment) against the oracle.

Each batch is replayed by the oracle in the reported commit order: every read
of a committed transaction and every column of the final database (including
the inserted orders, new-order flags and order lines) must match exactly; the
order-entry consistency conditions must hold; the deterministic scheme must
equal serial execution in transaction-id order.
"""
import numpy as np
import pytest

import oracle
from paper_2406_10158_gb300 import workload as wl

pytestmark = pytest.mark.gpu
SCHEMES = ["occ", "2pl", "2pl_wd", "to", "tictoc", "det", "det-dataflow", "det-gacco"]


def scheme_params(eng, scheme, **kw):
    """"det-dataflow" is the deterministic scheme run op by op in the execute
    kernel (order-entry batches otherwise take the per-record pass);
    "det-gacco" the same with every access to a record ordered."""
    if scheme == "det-dataflow":
        scheme, kw = "det", dict(kw, det_dataflow=1)
    elif scheme == "det-gacco":
        scheme, kw = "det", dict(kw, det_dataflow=2)
    return scheme, (eng.params(**kw) if kw else None)


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine
    return engine


def run_and_check(eng, W, n_txns, scheme, seed=5, lanes=None, by_name_frac=0.0):
    db0, batch, cap = wl.order_entry(seed=seed, W=W, n_txns=n_txns, by_name_frac=by_name_frac)
    with eng.Database("oe", n_warehouses=W, order_cap=cap, max_ops_per_txn=33,
                      max_batch_txns=n_txns, max_batch_ops=batch.n_ops) as db:
        db.load_oe(db0)
        # one lane per txn stages 32 txns x 33 ops per warp: one warp per block
        kw = dict(lanes_per_txn=lanes, warps_per_block=1 if lanes == 1 else 8) if lanes else {}
        name = scheme
        scheme, p = scheme_params(eng, scheme, **kw)
        res, reads, stats = db.run(scheme, batch, p, timeout_s=300)
        final = db.read_oe()
    assert stats["committed"] == n_txns and stats["device_error"] == 0, stats
    rep = oracle.oe_replay_check(db0, final, W, cap, batch, res, reads)
    assert rep["ok"], (scheme, rep)
    assert oracle.oe_consistency(final, W, cap) == 0
    if name.startswith("det"):
        ref, ref_reads = oracle.oe_serial(db0, W, cap, batch)
        assert np.array_equal(res["commit_order"], np.arange(n_txns))
        assert all(np.array_equal(ref[c], final[c]) for c in wl.OE_COLUMNS)
        assert np.array_equal(ref_reads, reads)
    return stats


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("W", [1, 8])
def test_order_entry_small(eng, scheme, W):
    run_and_check(eng, W, 1 << 13, scheme)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("W", [1, 8])
def test_order_entry_payment_by_last_name(eng, scheme, W):
    """60% of the payments name their customer by last name (TPC-C's share):
    the engine resolves each through its per-district sorted index before the
    transaction runs, and the history, replayed by the oracle (which picks
    the customer by scanning the district), matches exactly."""
    _, batch, _ = wl.order_entry(seed=5, W=W, n_txns=1 << 13, by_name_frac=0.6)
    assert (batch.ops["kind"] == wl.OE_C_PAY_BY_NAME).sum() > 1000
    run_and_check(eng, W, 1 << 13, scheme, by_name_frac=0.6)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_order_entry_lane_widths(eng, scheme):
    for lanes in (1, 4, 32):
        run_and_check(eng, 2, 4096, scheme, seed=11, lanes=lanes)


def test_order_entry_rejects_malformed(eng):
    W = 1
    db0, batch, cap = wl.order_entry(seed=3, W=W, n_txns=64)
    ops = batch.ops.copy()
    txns = batch.txns
    pay = np.nonzero(txns["type"] == wl.TXN_PAYMENT)[0][:2]
    no = np.nonzero(txns["type"] == wl.TXN_NEW_ORDER)[0][:1]
    ops["key"][txns["first_op"][pay[0]]] = W                 # warehouse out of range
    ops["kind"][txns["first_op"][pay[1]] + 1] = wl.OE_C_PAY  # wrong op layout
    ops["kind"][txns["first_op"][no[0]] + 3] = wl.OE_S_NEWORDER
    # payments by a name nobody has and by a district out of range
    pay2 = np.nonzero(txns["type"] == wl.TXN_PAYMENT)[0][2:4]
    for t, (key, name) in zip(pay2, [(3, 1000), (10 * W, 5)]):
        f = int(txns["first_op"][t]) + 2
        ops["kind"][f], ops["key"][f], ops["aux"][f] = wl.OE_C_PAY_BY_NAME, key, name
    bad_ids = [pay[0], pay[1], no[0], pay2[0], pay2[1]]
    bad = wl.KVBatch(txns=txns, ops=ops, operands=batch.operands)
    with eng.Database("oe", n_warehouses=W, order_cap=cap, max_ops_per_txn=33,
                      max_batch_txns=64, max_batch_ops=batch.n_ops) as db:
        for name in SCHEMES:
            db.load_oe(db0)
            scheme, p = scheme_params(eng, name)
            res, reads, stats = db.run(scheme, bad, p)
            st = res["status"]
            assert (st[bad_ids] == oracle.ST_INVALID).all(), name
            assert (np.delete(st, bad_ids) == oracle.ST_COMMITTED).all(), name


@pytest.mark.slow
@pytest.mark.parametrize("W", [1, 8, 64])
def test_order_entry_full_size(eng, W):
    """2^18 txns, 50/50 NewOrder/Payment, every scheme (the paper's TPC-C shape)."""
    for scheme in ["occ", "2pl", "2pl_wd", "to", "tictoc", "det"] + \
            (["det-dataflow", "det-gacco"] if W > 1 else []):
        run_and_check(eng, W, 1 << 18, scheme, seed=wl.SEEDS[2])
    # and with 60% of the payments by last name
    for scheme in ["occ", "to", "det"]:
        run_and_check(eng, W, 1 << 18, scheme, seed=wl.SEEDS[2], by_name_frac=0.6)
