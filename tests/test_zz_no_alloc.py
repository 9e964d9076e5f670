"""The allocation-free deterministic entry point matches the regular one.

gcc_det_execute_noalloc is for callers that cannot allocate device memory
(their device memory is reserved up front by another allocator, or they run
a latency-critical loop where cudaMalloc's implicit synchronisation is not
acceptable): it keeps its scratch in a static device array instead.  Here it
runs the same batches as gcc_execute with the deterministic scheme on a
database holding the same table, twice in a row, and every read value,
transaction result and table word must agree with that call and with the
oracle's serial execution in transaction-id order.  The test allocates its own
buffers with torch; the entry point itself allocates nothing.
"""
import ctypes

import numpy as np
import pytest

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


def _dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)).cuda()


def _noalloc(eng, lib, d_table, nrec, nf, fb, batch, torch, max_ops=16):
    """One call of the allocation-free entry point; returns its results and
    reads as device byte tensors."""
    d_txns, d_ops, d_opd = _dev(batch.txns, torch), _dev(batch.ops, torch), \
        _dev(batch.operands, torch)
    n_res = torch.zeros(max(1, batch.n_txns) * 16, dtype=torch.uint8, device="cuda")
    n_reads = torch.zeros(max(1, batch.n_ops) * 16, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rc = lib.gcc_det_execute_noalloc(d_table.data_ptr(), nrec, nf, fb, d_txns.data_ptr(),
                                     batch.n_txns, d_ops.data_ptr(), d_opd.data_ptr(),
                                     batch.n_ops, max_ops, n_res.data_ptr(),
                                     n_reads.data_ptr(), None)
    assert rc == 0, eng.gcc_last_error()
    torch.cuda.synchronize()
    return n_res, n_reads


@pytest.mark.parametrize("field_bytes", [8, 16])
def test_noalloc_matches_regular_entry_point_twice(eng, field_bytes):
    """Two batches in a row on one table: the allocation-free call, the
    regular deterministic call on a database holding the same table, and the
    oracle's serial execution in id order agree on every read, result and
    table word after each batch."""
    import oracle
    import torch
    nrec, nf = 65536, 8
    if field_bytes == 8:
        table = wl.kv_table_splitmix(wl.SEEDS[0], nrec, nf)
    else:
        table = wl.kv_table_bytes(wl.SEEDS[0], nrec, nf)
    batches = [wl.kv_batch(s, nrec=nrec, nfields=nf, n_txns=4096, ops_per_txn=16,
                           read_ratio=0.5, theta=0.9, field_bytes=field_bytes)
               for s in (31, 32)]
    lib = eng.load()
    d_table = _dev(table, torch)
    expect = table
    with eng.Database("kv", n_records=nrec, n_fields=nf, field_bytes=field_bytes,
                      max_batch_txns=4096) as db:
        db.load_kv(table)
        for batch in batches:
            d_txns, d_ops, d_opd = _dev(batch.txns, torch), _dev(batch.ops, torch), \
                _dev(batch.operands, torch)
            r_res = torch.zeros(batch.n_txns * 16, dtype=torch.uint8, device="cuda")
            r_reads = torch.zeros(batch.n_ops * 16, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()          # copies and fills done before other streams run
            # regular entry point (on the database's own stream)
            db.execute("det", d_txns, d_ops, d_opd, batch.n_txns, batch.n_ops, r_res, r_reads)
            # allocation-free entry point on the caller's own table copy
            n_res, n_reads = _noalloc(eng, lib, d_table, nrec, nf, field_bytes, batch, torch)
            res = n_res.cpu().numpy().view(wl.RESULT_DTYPE)
            assert (res["status"] == 1).all()
            assert np.array_equal(res["commit_order"], np.arange(batch.n_txns))
            assert torch.equal(n_res, r_res)
            assert torch.equal(n_reads, r_reads)
            regular_table = db.read_kv()
            mine = d_table.cpu().numpy().view(np.uint64).reshape(table.shape)
            assert np.array_equal(mine, regular_table)
            expect, ref_reads = oracle.serial(expect, batch)
            assert np.array_equal(mine, expect)
            assert np.array_equal(n_reads.cpu().numpy().view(np.uint64).reshape(-1, 2),
                                  ref_reads)


def test_noalloc_out_of_range_key_at_the_record_limit(eng):
    """At the 65,536-record limit (a power of two) an op whose key is out of
    range sits between two writers of record 0: its transaction comes back
    INVALID, and the two writers commit in id order with nothing left
    waiting."""
    import oracle
    import torch
    nrec, nf = 65536, 2
    table = wl.kv_table_splitmix(7, nrec, nf)
    batch = wl.kv_batch_from_lists([
        [(0, 0, 1, 5, 0)],
        [(nrec, 0, 1, 0, 0), (0, 1, 1, 2, 0)],
        [(0, 0, 1, 7, 0), (1, 1, 0, 0, 0)],
    ])
    lib = eng.load()
    d_table = _dev(table, torch)
    n_res, n_reads = _noalloc(eng, lib, d_table, nrec, nf, 8, batch, torch)
    res = n_res.cpu().numpy().view(wl.RESULT_DTYPE)
    assert res["status"].tolist() == [1, 3, 1]
    assert res["commit_order"][[0, 2]].tolist() == [0, 1]
    ref_final, ref_reads = oracle.serial(table, batch, order=[0, 2])
    mine = d_table.cpu().numpy().view(np.uint64).reshape(table.shape)
    assert np.array_equal(mine, ref_final)
    reads = n_reads.cpu().numpy().view(np.uint64).reshape(-1, 2)
    assert np.array_equal(reads[[0, 3, 4]], ref_reads[[0, 3, 4]])


def test_noalloc_rejects_oversized_batches(eng):
    import torch
    lib = eng.load()
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    rc = lib.gcc_det_execute_noalloc(p, 65537, 1, 8, p, 1, p, p, 1, 16, p, p, None)
    assert rc == 6 and "65536" in eng.gcc_last_error()
    rc = lib.gcc_det_execute_noalloc(p, 16, 1, 8, p, 1, p, p, 65537, 16, p, p, None)
    assert rc == 6
