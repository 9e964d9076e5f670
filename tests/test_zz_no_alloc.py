"""The allocation-free deterministic entry point matches the regular one.

gcc_det_execute_noalloc is for callers that cannot allocate device memory
(their device memory is reserved up front by another allocator, or they run
a latency-critical loop where cudaMalloc's implicit synchronisation is not
acceptable): it keeps its scratch in a static device array instead.  Here it
runs the same batches as gcc_execute with the deterministic scheme on a
database holding the same table, twice in a row, and every read value,
transaction result and table word must agree.  The test allocates its own
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


def test_noalloc_matches_regular_entry_point_twice(eng):
    import torch
    nrec, nf = 65536, 8
    table = wl.kv_table_splitmix(wl.SEEDS[0], nrec, nf)
    batches = [wl.kv_batch(s, nrec=nrec, nfields=nf, n_txns=4096, ops_per_txn=16,
                           read_ratio=0.5, theta=0.9) for s in (31, 32)]
    lib = eng.load()
    d_table = _dev(table, torch)
    with eng.Database("kv", n_records=nrec, n_fields=nf, field_bytes=8,
                      max_batch_txns=4096) as db:
        db.load_kv(table)
        for batch in batches:
            d_txns, d_ops, d_opd = _dev(batch.txns, torch), _dev(batch.ops, torch), \
                _dev(batch.operands, torch)
            r_res = torch.zeros(batch.n_txns * 16, dtype=torch.uint8, device="cuda")
            r_reads = torch.zeros(batch.n_ops * 16, dtype=torch.uint8, device="cuda")
            n_res = torch.zeros_like(r_res)
            n_reads = torch.zeros_like(r_reads)
            torch.cuda.synchronize()          # copies and fills done before other streams run
            # regular entry point (on the database's own stream)
            db.execute("det", d_txns, d_ops, d_opd, batch.n_txns, batch.n_ops, r_res, r_reads)
            # allocation-free entry point on the caller's own table copy
            rc = lib.gcc_det_execute_noalloc(d_table.data_ptr(), nrec, nf, 8, d_txns.data_ptr(),
                                             batch.n_txns, d_ops.data_ptr(), d_opd.data_ptr(),
                                             batch.n_ops, 16, n_res.data_ptr(),
                                             n_reads.data_ptr(), None)
            assert rc == 0, eng.gcc_last_error()
            torch.cuda.synchronize()
            res = n_res.cpu().numpy().view(wl.RESULT_DTYPE)
            assert (res["status"] == 1).all()
            assert np.array_equal(res["commit_order"], np.arange(batch.n_txns))
            assert torch.equal(n_res, r_res)
            assert torch.equal(n_reads, r_reads)
            regular_table = db.read_kv()
            mine = d_table.cpu().numpy().view(np.uint64).reshape(nf, nrec)
            assert np.array_equal(mine, regular_table)


def test_noalloc_rejects_oversized_batches(eng):
    import torch
    lib = eng.load()
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    rc = lib.gcc_det_execute_noalloc(p, 65537, 1, 8, p, 1, p, p, 1, 16, p, p, None)
    assert rc == 6 and "65536" in eng.gcc_last_error()
    rc = lib.gcc_det_execute_noalloc(p, 16, 1, 8, p, 1, p, p, 65537, 16, p, p, None)
    assert rc == 6
