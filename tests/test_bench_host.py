"""Host arithmetic behind the benchmark's reported bounds."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2406_10158_gb300 import workload as wl  # noqa: E402


def _batch():
    # txn 0: read key 3, add key 5; txn 1: add key 5, read key 7; txn 2: add key 5
    return wl.kv_batch_from_lists([
        [(3, 0, wl.OP_READ, 0, 0), (5, 1, wl.OP_ADD, 4, 0)],
        [(5, 0, wl.OP_ADD, -2, 0), (7, 0, wl.OP_READ, 0, 0)],
        [(5, 0, wl.OP_ADD, 9, 0)],
    ], field_bytes=16)


def test_algorithmic_bytes_count_each_op_once():
    b = _batch()
    alg = bench.algorithmic_bytes(b)
    assert (alg["reads"], alg["writes"]) == (2, 3)
    assert alg["bytes"] == 3 * 24 + 2 * 56 + 3 * 88


def test_sector_bytes():
    b = _batch()
    s = bench.sector_bytes(b)
    assert s["random"] == 5 * 64 + 3 * 64
    assert s["stream"] == 3 * 24 + 5 * 8 + 3 * 16 + 5 * 16


def test_hot_record_counts():
    c = bench.hot_record_counts(_batch())
    assert c == {"max_accesses": 3, "max_writes": 3}


def test_hot_record_of_a_zipf_batch_matches_its_histogram():
    b = wl.kv_batch(7, nrec=1 << 12, nfields=2, n_txns=2048, theta=0.9, read_ratio=0.5)
    keys = b.ops["key"].astype(np.int64)
    w = b.ops["kind"] == wl.OP_ADD
    c = bench.hot_record_counts(b)
    assert c["max_accesses"] == np.bincount(keys).max()
    assert c["max_writes"] == np.bincount(keys[w]).max()
    assert c["max_writes"] <= c["max_accesses"]


def test_captured_traffic_only_while_the_kernel_is_unchanged(monkeypatch):
    """A captured DRAM figure is reported only for its own workload and only
    while the digest of the kernel sources equals the one it was taken on."""
    key = ("occ", 1 << 24, 1 << 20, 0.8, 0.5, 0, 0)
    digest = bench.kernel_sources_digest()
    assert len(digest) == 16 and digest == bench.kernel_sources_digest()
    monkeypatch.setattr(bench, "CAPTURED_TRAFFIC", {key: (4.0e9, digest)})
    assert bench.captured_traffic(key) == 4.0e9
    assert bench.captured_traffic(("occ", 1 << 24, 1 << 20, 0.6, 0.5, 0, 0)) is None
    assert bench.captured_traffic(("2pl", 1 << 24, 1 << 20, 0.8, 0.5, 0, 0)) is None
    monkeypatch.setattr(bench, "CAPTURED_TRAFFIC", {key: (4.0e9, "0" * 16)})
    assert bench.captured_traffic(key) is None


def test_oracle_timing_covers_the_whole_batch():
    table = wl.kv_table_splitmix(3, 512, 2)
    b = wl.kv_batch(4, nrec=512, nfields=2, n_txns=300, ops_per_txn=4)
    v, info = bench.time_oracle(table, b, 0.0)
    assert info["txns"] == b.n_txns and info["repeats"] == 1 and v > 0


def test_host_info_names_cores_and_model():
    h = bench.host_info()
    assert h["nproc"] == os.cpu_count() and h["nproc"] >= 1
    assert isinstance(h["cpu"], str) and h["cpu"]
    assert h["machine"]


def test_order_entry_bytes_by_procedure():
    """A NewOrder of L lines moves 224 + 184 L useful bytes, a Payment 272:
    per transaction 24, then its ops and inserts (the byte table's sums)."""
    _, oe, _ = wl.order_entry(seed=3, W=2, n_txns=400)
    got = bench.oe_algorithmic_bytes(oe)
    is_no = oe.txns["type"] == wl.TXN_NEW_ORDER
    lines = (oe.txns["n_ops"][is_no].astype(np.int64) - 3) // 2
    want = int((224 + 184 * lines).sum()) + 272 * int((~is_no).sum())
    assert got["bytes"] == want
    assert got["new_orders"] == int(is_no.sum()) and got["lines"] == int(lines.sum())
    assert 900 < got["per_txn"] < 1400            # about 1.2 KB at 50/50 and 10 lines


def test_served_latency_is_reported_at_the_highest_sustained_rate():
    rows = [{"offered_txn_per_s": 1e5, "committed_txn_per_s": 1.0e5, "p99_latency_us": 300},
            {"offered_txn_per_s": 1e7, "committed_txn_per_s": 0.99e7, "p99_latency_us": 4000},
            {"offered_txn_per_s": 1e8, "committed_txn_per_s": 2.4e7, "p99_latency_us": 3e5}]
    assert bench.sustained_rate(rows)["offered_txn_per_s"] == 1e7
    rows[1]["committed_txn_per_s"] = 0.9e7            # 10^7 no longer sustained
    assert bench.sustained_rate(rows)["offered_txn_per_s"] == 1e5
    # nothing sustained: the highest committed rate
    assert bench.sustained_rate(rows[2:])["offered_txn_per_s"] == 1e8
