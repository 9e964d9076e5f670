"""GPU parity of the batched form: several independent key-value batches in
one persistent launch (plain and as a replayed CUDA graph).  Every batch is
replayed by the oracle in its reported commit order against its own database.
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)).cuda()


def make_set(eng, n_db=6, seed=3, spec=None):
    import torch
    if spec is None:
        spec = wl.batched_kv(seed, n_db=n_db, rec_bits=(10, 14), txn_range=(50, 3000),
                             ops_range=(4, 64), theta=0.8)
    entries, dbs = [], []
    for (nrec, table, batch) in spec:
        db = eng.Database("kv", n_records=nrec, n_fields=8, field_bytes=8, max_ops_per_txn=64,
                          max_batch_txns=batch.n_txns, max_batch_ops=batch.n_ops)
        db.load_kv(table)
        res = torch.zeros(batch.n_txns * 16, dtype=torch.uint8, device="cuda")
        reads = torch.zeros(batch.n_ops * 16, dtype=torch.uint8, device="cuda")
        entries.append((db, _dev(batch.txns), batch.n_txns, _dev(batch.ops), _dev(batch.operands),
                        batch.n_ops, res, reads))
        dbs.append((db, table, batch, res, reads))
    torch.cuda.synchronize()
    return entries, dbs


def check_all(eng, plan, dbs, states, det=False):
    import torch
    torch.cuda.synchronize()
    new_states = []
    for i, ((db, _, batch, res, reads), state) in enumerate(zip(dbs, states)):
        r = res.cpu().numpy().view(wl.RESULT_DTYPE)
        rd = reads.cpu().numpy().view(np.uint64).reshape(-1, 2)
        final = db.read_kv()
        st = plan.stats(i)
        assert st["committed"] == batch.n_txns, (i, st)
        rep = oracle.replay_check(state, final, batch, r, rd)
        assert rep["ok"], (i, rep)
        if det:                           # the deterministic outcome: id order
            assert np.array_equal(r["commit_order"], np.arange(batch.n_txns)), i
        new_states.append(final)
    return new_states


@pytest.mark.parametrize("scheme", ["occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc", "det"])
def test_batched_form_replays(eng, scheme):
    entries, dbs = make_set(eng)
    plan = eng.MultiPlan(scheme, entries, eng.params(backoff_cap_ns=16_000_000))
    states = [t for (_, t, _, _, _) in dbs]
    plan.launch(use_graph=False)
    states = check_all(eng, plan, dbs, states, det=scheme == "det")
    for _ in range(2):                    # graph capture, then a replay
        plan.launch(use_graph=True)
        states = check_all(eng, plan, dbs, states, det=scheme == "det")
    plan.close()
    for (db, *_rest) in dbs:
        db.close()


@pytest.mark.slow
def test_batched_form_full_size(eng):
    """The batched workload as the benchmark builds it: 64 databases of
    2^16..2^22 records (log-uniform) x 8 u64 fields, batches of 1,000 ..
    262,144 txns of 4..64 ops at Zipf 0.8, in one graph-replayed plan per
    scheme (every scheme); every database's history replays exactly."""
    spec = wl.batched_kv(wl.SEEDS[3], n_db=64)
    entries, dbs = make_set(eng, spec=spec)
    states = [t for (_, t, _, _, _) in dbs]
    for scheme in ("occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc", "det"):
        plan = eng.MultiPlan(scheme, entries, eng.params(backoff_cap_ns=16_000_000))
        plan.launch(use_graph=True)
        states = check_all(eng, plan, dbs, states, det=scheme == "det")
        plan.close()
    for (db, *_rest) in dbs:
        db.close()


def test_batched_form_guards_scheme_changes(eng):
    import torch
    entries, dbs = make_set(eng, n_db=2, seed=9)
    plan = eng.MultiPlan("occ", entries)
    plan.launch(use_graph=True)
    torch.cuda.synchronize()
    db, _, batch, *_ = dbs[0]
    db.run("2pl", batch)                  # leaves 2PL-compatible words: OCC may resume
    plan.launch(use_graph=True)
    torch.cuda.synchronize()              # the plan's stream and the database's are separate
    db.run("to", batch)                   # 16-byte TO words: the plan must refuse
    with pytest.raises(eng.GCCError):
        plan.launch(use_graph=True)
    plan.close()
    for (d, *_rest) in dbs:
        d.close()


def test_autotune_picks_a_valid_faster_point(eng):
    import torch
    nrec = 1 << 14
    table = wl.kv_table_splitmix(4, nrec, 8)
    batch = wl.kv_batch(5, nrec=nrec, nfields=8, n_txns=8192, theta=0.8)
    with eng.Database("kv", n_records=nrec, n_fields=8, field_bytes=8, max_batch_txns=8192) as db:
        db.load_kv(table)
        tx, op, od = _dev(batch.txns), _dev(batch.ops), _dev(batch.operands)
        res = torch.zeros(batch.n_txns * 16, dtype=torch.uint8, device="cuda")
        reads = torch.zeros(batch.n_ops * 16, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        space = eng.tune_space(lanes=(4, 16), warps=(4, 8), caps=(65536, 1000000), steps=2)
        best, rep = eng.gcc_autotune(db.handle, "occ", tx.data_ptr(), batch.n_txns, op.data_ptr(),
                                     od.data_ptr(), batch.n_ops, res.data_ptr(), reads.data_ptr(),
                                     space)
        assert rep["points"] == 8
        assert rep["best_txn_per_s"] >= rep["default_txn_per_s"] > 0
        assert best.lanes_per_txn in (4, 16) or rep["best_txn_per_s"] == rep["default_txn_per_s"]
        # the chosen parameters run a batch that replays exactly
        state = db.read_kv()
        r, rd, st = db.run("occ", batch, best)
        assert oracle.replay_check(state, db.read_kv(), batch, r, rd)["ok"]
