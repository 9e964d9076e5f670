"""Memory-system probes behind the rooflines (gcc_probe_memory)."""
import math

import numpy as np
import pytest

from paper_2406_10158_gb300 import engine as eng
from paper_2406_10158_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return eng


def test_probe_figures_are_physical(built):
    m = eng.gcc_probe_memory(0)
    for k, v in m.items():
        for x in (v if isinstance(v, list) else [v]):
            assert math.isfinite(x) and x > 0, (k, v)
    # a line in L2 answers sooner than one in HBM; one word's atomics are a
    # serial resource, distinct words are not
    assert m["l2_load_ns"] < m["hbm_load_ns"]
    assert m["occ_cycle_ns"] <= m["occ_cycle_busy_ns"]
    assert m["add_same_gops"] < m["cas_distinct_gops"]
    # a commit on one record costs at least one hand-off of its lock
    assert m["occ_cycle_ns"] > 0.5 * m["lock_handoff_ns"]
    assert m["contenders"] == 8 * m["sm_count"]
    # the random-sector ceiling is the best of the in-flight sweep
    assert m["gather32_gbs"] == max(m["gather32_by_inflight_gbs"])
    assert m["gather32_best_inflight"] in (4, 8, 16)
    # one link of the commit chain holds a CAS, an acquire-release atomic
    # (itself at least a fence) and a release store
    assert m["atomic_acq_rel_ns"] > 0.5 * m["fence_ns"]
    assert m["occ_link_ns"] > m["atomic_acq_rel_ns"]
    assert m["occ_link_ns"] > m["l2_cas_ns"]
    assert m["occ_link_max_ns"] >= m["occ_link_ns"]


def test_execute_kernel_counts_its_atomics(built):
    """The execute kernel's own atomic count: under OCC every committed write
    takes at least one lock CAS, and with no contention (disjoint keys, one
    attempt each) nothing is retried, so the count stays within a few
    atomics per op."""
    nrec, nf = 1 << 14, 2
    table = wl.kv_table_splitmix(3, nrec, nf)
    batch = wl.disjoint_kv(4, n_txns=512, nrec=nrec, nfields=nf, ops_per_txn=16)
    with eng.Database("kv", n_records=nrec, n_fields=nf, field_bytes=8,
                      max_batch_txns=512) as db:
        db.load_kv(table)
        for scheme in ("occ", "2pl", "to"):
            res, reads, st = db.run(scheme, batch)
            assert st["committed"] == batch.n_txns and st["aborts"] == 0, (scheme, st)
            writes = int(np.count_nonzero(batch.ops["kind"] == wl.OP_ADD))
            assert writes <= st["atomics"] <= 3 * batch.n_ops + 2 * batch.n_txns, (scheme, st)
