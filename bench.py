#!/usr/bin/env python3
"""Benchmark: committed transactions/s and abort rate of one GPU batch.

A step is one batch of 2^20 key-value transactions (16 ops each over 2^24
records x 10 fields in 16-byte slots, Zipfian keys) through the whole
execution path: control-word setup, [deterministic preprocessing], the
execute kernel and the dense commit ranks.  Inputs are resident in HBM when
the timed region starts; the table (2.5 GiB) and the batch (400 MB) are
larger than L2, so no flush is needed between steps.

The headline line is OCC at theta 0.8, read ratio 0.5; ``schemes`` adds the
same workload under every scheme.  ``--impl reference`` times the CPU oracle
(single-threaded serial execution) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "committed txns/s + abort rate on 1 GB300 vs plain launch; p99 commit latency"
SCHEMES = ["occ", "2pl", "2pl_wd", "to", "tictoc", "mvcc", "det"]


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1,
                   help="GPUs (one replica each; under torchrun, the world size)")
    p.add_argument("--steps", type=int, default=20, help="timed batches")
    p.add_argument("--warmup", type=int, default=3, help="untimed batches before them")
    p.add_argument("--impl", choices=["ours", "reference"], default="ours",
                   help="ours: the engine; reference: the CPU oracle on the same workload")
    p.add_argument("--scheme", default="occ", choices=SCHEMES, help="scheme of the headline line")
    p.add_argument("--theta", type=float, default=0.8, help="Zipf skew of the keys (0: uniform)")
    p.add_argument("--read-ratio", type=float, default=0.5, help="share of READ ops")
    p.add_argument("--records", type=int, default=1 << 24, help="key-value records")
    p.add_argument("--txns", type=int, default=1 << 20, help="transactions per batch")
    p.add_argument("--lanes", type=int, default=0, help="lanes per transaction (0 = default)")
    p.add_argument("--warps", type=int, default=0, help="warps per block (0 = default)")
    p.add_argument("--no-schemes", action="store_true", help="skip the per-scheme lines")
    p.add_argument("--scheme-steps", type=int, default=3, help="timed batches per scheme line")
    p.add_argument("--scheme-deadline-s", type=float, default=20.0,
                   help="kernel deadline for the per-scheme lines")
    p.add_argument("--no-e2e", action="store_true",
                   help="skip the end-to-end measurement through submit/wait")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="about how long the CPU baseline runs")
    p.add_argument("--seed", type=int, default=0x5EED0002, help="workload seed")
    p.add_argument("--form", choices=["plain", "batched", "served", "sweep"], default="plain",
                   help="plain: one batch per launch (the default line); batched: 64 "
                        "databases in one persistent launch vs 64 plain launches; served: "
                        "continuous batching of a Poisson trace vs plain per-batch launches; "
                        "sweep: every scheme across the key-value contention levels and the "
                        "order-entry warehouse counts")
    p.add_argument("--check", action="store_true",
                   help="sweep: replay every cell's batch on the CPU oracle (slow)")
    p.add_argument("--sweep-parts", default="kv,hotspot,oe",
                   help="sweep form: which parts to run (kv, hotspot, oe), comma-separated")
    p.add_argument("--n-db", type=int, default=64, help="batched form: databases")
    p.add_argument("--rates", default="1e5,1e6,1e7,1e8",
                   help="served form: offered rates (txn/s), comma-separated")
    p.add_argument("--requests", type=int, default=10_000_000,
                   help="served form: most requests per rate (each rate runs at most 10 s "
                        "of arrivals)")
    p.add_argument("--kv-scheme", default="det", choices=SCHEMES, help="served form: key-value lane")
    p.add_argument("--served-depth", type=int, default=4,
                   help="served form: batches in flight per lane (1..8)")
    p.add_argument("--served-delay-us", type=int, default=400,
                   help="served form: longest wait of a batch's oldest request before launch")
    p.add_argument("--served-max-batch", type=int, default=1 << 14,
                   help="served form: transactions per batch at most")
    p.add_argument("--oe-scheme", default="det", choices=SCHEMES, help="served form: order-entry lane")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the GPU works."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, p in rows for n, v in zip(names, p[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def algorithmic_bytes(batch) -> dict:
    """Bytes the method must move per batch (useful bytes): per transaction
    its 8-byte descriptor and 16-byte result; per READ op 8 descriptor + 8
    control word + 16 slot + 8 control-word revalidation + 16 value out; per
    read-modify-write op 8 descriptor + 16 operand + 16 slot read + 16 slot
    write + 8 lock + 8 unlock/version + 16 value out."""
    from paper_2406_10158_gb300 import workload as wl
    n_w = int(np.count_nonzero(batch.ops["kind"] == wl.OP_ADD))
    n_r = batch.n_ops - n_w
    per_txn = 8 + 16
    total = batch.n_txns * per_txn + n_r * 56 + n_w * 88
    return {"bytes": total, "reads": n_r, "writes": n_w, "per_txn": total / max(1, batch.n_txns)}


def mvcc_algorithmic_bytes(batch) -> dict:
    """algorithmic_bytes plus, per read-modify-write, the version it makes:
    a 28-byte store entry (timestamp, link, field, 16-byte value) written at
    commit and read back once when the batch's versions go into the table."""
    from paper_2406_10158_gb300 import workload as wl
    base = algorithmic_bytes(batch)
    n_w = int(np.count_nonzero(batch.ops["kind"] == wl.OP_ADD))
    total = base["bytes"] + n_w * 2 * 28
    return {"bytes": total, "per_txn": total / max(1, batch.n_txns)}


# Useful bytes of one order-entry op by kind (8-byte descriptor, 16-byte value
# out; control word read + revalidated, or locked + unlocked, 8 + 8; the int64
# columns the procedure reads and writes; 16-byte operand where it has one).
OE_OP_BYTES = {
    "w_read": 8 + 16 + 16 + 8,                        # w_tax
    "d_neworder": 8 + 16 + 16 + 8 + 8 + 8,            # d_next_o_id r/w, d_tax
    "c_read": 8 + 16 + 16 + 8 + 8,                    # c_discount, c_balance
    "i_read": 8 + 16 + 8,                             # i_price, no control word
    "s_neworder": 8 + 16 + 16 + 16 + 4 * 16,          # s_quantity, s_order_cnt, s_ytd,
                                                      # s_remote_cnt read and written
    "w_pay": 8 + 16 + 16 + 16 + 16,                   # w_ytd r/w
    "d_pay": 8 + 16 + 16 + 16 + 16,                   # d_ytd r/w
    "c_pay": 8 + 16 + 16 + 16 + 3 * 16,               # c_balance, c_payment_cnt,
}                                                     # c_ytd_payment read and written
OE_ORDER_INSERT = 4 * 8                               # o_c_id, o_ol_cnt, o_all_local, no_flag
OE_LINE_INSERT = 4 * 8                                # ol_i_id, ol_supply_w_id, ol_quantity,
                                                      # ol_amount


def oe_algorithmic_bytes(batch) -> dict:
    """Useful bytes of an order-entry batch: per transaction its 8-byte
    descriptor and 16-byte result, per op OE_OP_BYTES of its kind, and the
    rows a NewOrder inserts (its order and new-order row, and one row per
    line)."""
    from paper_2406_10158_gb300 import workload as wl
    kinds = {wl.OE_W_READ: "w_read", wl.OE_D_NEWORDER: "d_neworder", wl.OE_C_READ: "c_read",
             wl.OE_I_READ: "i_read", wl.OE_S_NEWORDER: "s_neworder", wl.OE_W_PAY: "w_pay",
             wl.OE_D_PAY: "d_pay", wl.OE_C_PAY: "c_pay"}
    count = np.bincount(batch.ops["kind"].astype(np.int64), minlength=32)
    total = batch.n_txns * (8 + 16)
    for k, name in kinds.items():
        total += int(count[k]) * OE_OP_BYTES[name]
    total += int(count[wl.OE_D_NEWORDER]) * OE_ORDER_INSERT + int(count[wl.OE_S_NEWORDER]) * OE_LINE_INSERT
    return {"bytes": total, "new_orders": int(count[wl.OE_D_NEWORDER]),
            "payments": int(count[wl.OE_W_PAY]), "lines": int(count[wl.OE_S_NEWORDER]),
            "per_txn": total / max(1, batch.n_txns)}


def hot_record_counts(batch) -> dict:
    """Accesses and writes of the most accessed / most written record."""
    from paper_2406_10158_gb300 import workload as wl
    keys = batch.ops["key"].astype(np.int64)
    w = batch.ops["kind"] == wl.OP_ADD
    acc = np.bincount(keys)
    wr = np.bincount(keys[w]) if w.any() else np.zeros(1, np.int64)
    return {"max_accesses": int(acc.max()), "max_writes": int(wr.max())}


def sector_bytes(batch) -> dict:
    """DRAM bytes at 32-byte sector granularity: every op touches its
    control word's sector and its slot's sector at random (plus a write-back
    of each for a read-modify-write); descriptors, operands, results and read
    values stream sequentially."""
    from paper_2406_10158_gb300 import workload as wl
    n_w = int(np.count_nonzero(batch.ops["kind"] == wl.OP_ADD))
    n = batch.n_ops
    random = n * 64 + n_w * 64
    stream = batch.n_txns * 24 + n * 8 + n_w * 16 + n * 16
    return {"random": random, "stream": stream, "per_txn": (random + stream) / max(1, batch.n_txns)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, bytes) of one
# execute-kernel launch from an ncu capture, keyed by workload (scheme,
# records, txns, theta, read ratio, lanes, warps) and stored with the digest
# of the kernel sources it was taken on: a capture counts only while the
# sources are unchanged (kernel_sources_digest), and the line reports null
# otherwise.
CAPTURED_TRAFFIC = {
    # the default line's workload: ncu --metrics dram__bytes_read.sum,
    # dram__bytes_write.sum,gpu__time_duration.sum (one pass), second
    # execute-kernel launch of `bench.py --steps 1 --warmup 1 --no-schemes
    # --no-e2e --no-cpu`: 3.51 GB read + 0.721 GB written
    ("occ", 1 << 24, 1 << 20, 0.8, 0.5, 0, 0): (4_231_620_000, "0f37401239eac6cc"),
}


def kernel_sources_digest() -> str:
    """SHA-256 (first 16 hex digits) over the engine's CUDA sources and the
    public header, in file-name order."""
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2406_10158_gb300", "csrc", "*.cu*")) +
                   glob.glob(os.path.join(ROOT, "include", "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(key):
    """The captured DRAM bytes per launch for this workload, or None when
    there is none or the kernel sources changed since it was taken."""
    got = CAPTURED_TRAFFIC.get(key)
    if got is None:
        return None
    value, digest = got
    return value if digest == kernel_sources_digest() else None


def replica_totals(dist, committed: float, elapsed: float, device=None):
    """Whole-job totals over replicas (one independent database and batch per
    rank): the committed transactions of all ranks and the slowest rank's
    elapsed time.  Without a process group, the local values."""
    if dist is None:
        return committed, elapsed
    import torch
    c = torch.tensor([float(committed)], dtype=torch.float64, device=device)
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(c.item()), float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_info() -> dict:
    """The host the CPU baseline ran on: its core count and CPU model."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            fields = {}
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
        model = fields.get("model name")
        if not model and "CPU part" in fields:   # Arm: implementer and part numbers
            model = f"implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(),
            "cpu": model or platform.processor() or "unknown"}


def time_oracle(table, batch, seconds: float):
    """Single-threaded serial execution (the CPU oracle) of the whole batch,
    in transaction-id order, repeated until about ``seconds`` have passed
    (at least once); returns (txn/s, details).  Each pass continues from the
    table the previous one left, so every pass does the full batch's work."""
    import oracle
    work = table.copy()
    done, t_total, reps = 0, 0.0, 0
    while t_total < seconds or reps == 0:
        t0 = time.perf_counter()
        oracle.serial_inplace(work, batch)
        t_total += time.perf_counter() - t0
        done += batch.n_txns
        reps += 1
    return done / t_total, {"txns": batch.n_txns, "repeats": reps, "seconds": round(t_total, 3)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2406_10158_gb300 import workload as wl
    table, batch = wl.ycsb_kv(args.seed, theta=args.theta, read_ratio=args.read_ratio,
                              nrec=args.records, n_txns=args.txns)
    import oracle
    # every step is the whole batch, serially in transaction-id order (the
    # deterministic scheme's outcome), continuing from the previous step's table
    work = table.copy()
    for _ in range(max(0, args.warmup)):
        oracle.serial_inplace(work, batch)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.serial_inplace(work, batch)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = batch.n_txns * args.steps / total
    workload = config_dict(args)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "txn/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload,
            "cpu_baseline": {"value": value, "unit": "txn/s", "cores": 1, "kind": "oracle",
                             "sample": f"the whole batch of {batch.n_txns} txns per step, "
                                       "serial in transaction-id order",
                             "host": host_info()},
            "e2e": {"value": value, "unit": "txn/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def config_dict(args):
    return {"workload": f"kv 16B slots {args.records}x10, {args.txns} txns x 16 ops, "
                        f"zipf {args.theta}, read ratio {args.read_ratio}",
            "scheme": args.scheme, "records": args.records, "fields": 10, "slot_bytes": 16,
            "txns_per_batch": args.txns, "ops_per_txn": 16, "theta": args.theta,
            "read_ratio": args.read_ratio,
            "l2": "inputs larger than L2 (2.5 GiB table, 400 MB batch); no flush",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, dist):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine as eng
    from paper_2406_10158_gb300 import workload as wl

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    table, batch = wl.ycsb_kv(args.seed + rank, theta=args.theta, read_ratio=args.read_ratio,
                              nrec=args.records, n_txns=args.txns)
    db = eng.Database("kv", n_records=args.records, n_fields=10, field_bytes=16,
                      max_ops_per_txn=16, max_batch_txns=args.txns, device=dev)
    db.load_kv(table)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    t_txns = torch.from_numpy(batch.txns.view(np.uint8)).to(dev)
    t_ops = torch.from_numpy(batch.ops.view(np.uint8)).to(dev)
    t_operands = torch.from_numpy(batch.operands.view(np.uint8).reshape(-1)).to(dev)
    t_res = torch.empty(batch.n_txns * 16, dtype=torch.uint8, device=dev)
    t_reads = torch.empty(batch.n_ops * 16, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)       # input copies done before the engine's stream runs
    probe = eng.gcc_probe_memory(dev) if rank == 0 else None
    kw = {}
    if args.lanes:
        kw["lanes_per_txn"] = args.lanes
    if args.warps:
        kw["warps_per_block"] = args.warps
    prm = eng.params(**kw)

    prm_sweep = eng.params(**kw, deadline_ns=int(args.scheme_deadline_s * 1e9))

    def step(scheme, p=None):
        db.execute(scheme, t_txns, t_ops, t_operands, batch.n_txns, batch.n_ops, t_res, t_reads,
                   p or prm, sh)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    def timed(scheme, steps, warmup, p=None):
        for _ in range(warmup):
            step(scheme, p)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(scheme, p)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        hist = db.stage_history(steps)
        stats = db.last_stats()
        return ms, hist, stats

    with ClockSampler(dev) as clocks:
        ms, hist, stats = timed(args.scheme, args.steps, args.warmup)
        committed = stats["committed"]
        committed_all, ms_max = replica_totals(dist, committed * args.steps, ms, dev)
        value = committed_all / (ms_max / 1000.0)
        kernel_ms = statistics.mean(h["kernel_ms"] for h in hist)
        launches = sum(h["kernel_launches"] for h in hist)

        # per-scheme lines on the same workload
        schemes = {}
        if not args.no_schemes:
            for s in SCHEMES:
                sms, shist, sst = timed(s, args.scheme_steps, 1, prm_sweep)
                schemes[s] = {
                    "committed_txn_per_s": sst["committed"] * args.scheme_steps / (sms / 1000.0),
                    "abort_rate": sst["abort_rate"], "ms_per_batch": sms / args.scheme_steps,
                    "prep_ms": statistics.mean(h["prep_ms"] for h in shist),
                    "kernel_ms": statistics.mean(h["kernel_ms"] for h in shist),
                    "order_ms": statistics.mean(h["order_ms"] for h in shist),
                    "all_committed": sst["committed"] == batch.n_txns,
                }

        # end to end through the public API with host buffers
        e2e = None
        if not args.no_e2e:
            pin = lambda a: torch.from_numpy(a.view(np.uint8).reshape(-1)).pin_memory()
            h_txns, h_ops, h_opd = pin(batch.txns), pin(batch.ops), pin(batch.operands)
            h_res = torch.empty(batch.n_txns * 16, dtype=torch.uint8).pin_memory()
            h_reads = torch.empty(batch.n_ops * 16, dtype=torch.uint8).pin_memory()
            e2e_steps = max(3, min(args.steps, 10))

            def api_step():
                b = eng.gcc_txn_batch_submit(db.handle, args.scheme, h_txns.data_ptr(),
                                             batch.n_txns, h_ops.data_ptr(), h_opd.data_ptr(),
                                             batch.n_ops, False, prm, sh)
                st = eng.gcc_batch_wait(b, eng.WAIT_FOREVER, h_res.data_ptr(), h_reads.data_ptr())
                eng.gcc_batch_free(b)
                return st

            api_step()
            barrier()
            t0 = time.perf_counter()
            committed_e2e = 0
            for _ in range(e2e_steps):
                committed_e2e += api_step()["committed"]
            barrier()
            dt = time.perf_counter() - t0
            committed_e2e, dt = replica_totals(dist, committed_e2e, dt, dev)
            e2e = {"value": committed_e2e / dt, "unit": "txn/s",
                   "h2d_bytes_per_step": batch.n_txns * 8 + batch.n_ops * 24,
                   "d2h_bytes_per_step": batch.n_txns * 16 + batch.n_ops * 16,
                   "steps": e2e_steps, "api": "gcc_txn_batch_submit + gcc_batch_wait"}
    clock = clocks.summary()

    if rank != 0:
        db.close()
        return None

    alg = algorithmic_bytes(batch)
    peak, peak_kind = measured_peaks()
    achieved = alg["bytes"] / (kernel_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": captured_traffic((args.scheme, args.records, args.txns, args.theta,
                                             args.read_ratio, args.lanes, args.warps)),
                "kernel_sources": kernel_sources_digest(),
                "kernel": f"kv_exec_kernel<{args.scheme}>", "kernel_ms": round(kernel_ms, 4),
                "algorithmic_bytes_per_launch": alg["bytes"],
                "algorithmic_bytes_per_txn": round(alg["per_txn"], 1),
                "peak_kind": f"{peak_kind} hbm_gbs"}
    # the serial chain on the hottest record: every committed write to it is
    # one link, and one link costs at least one contended OCC commit cycle
    hot = hot_record_counts(batch)
    bound_ms = hot["max_writes"] * probe["occ_cycle_ns"] / 1e6
    sect = sector_bytes(batch)
    sect_gbs = (sect["random"] + sect["stream"]) / (kernel_ms / 1000.0) / 1e9
    link_ms = hot["max_writes"] * probe["occ_link_ns"] / 1e6
    contention = {
        "bound": "hot-record chain", "hot_record_writes": hot["max_writes"],
        "hot_record_accesses": hot["max_accesses"], "cycle_ns": round(probe["occ_cycle_ns"], 1),
        "cycle_kind": "measured gcc_probe_memory occ_cycle_ns (best over contender counts)",
        "bound_ms": round(bound_ms, 3), "kernel_ms": round(kernel_ms, 4),
        "frac": round(bound_ms / kernel_ms, 4),
        # second bound: one uncontended link of the engine's own commit
        # sequence per committed writer of the hottest record
        "link_ns": round(probe["occ_link_ns"], 1),
        "link_max_ns": round(probe["occ_link_max_ns"], 1),
        "link_kind": "measured gcc_probe_memory occ_link_ns (acquire, CAS, acq_rel timestamp, "
                     "validation load, store, release publish; one thread, least over eight "
                     "SM placements; link_max_ns the greatest)",
        "link_bound_ms": round(link_ms, 3), "link_frac": round(link_ms / kernel_ms, 4),
        # third bound: a bare hand-off per link, two dependent L2 atomics (the
        # lock and the publish) and nothing else
        "handoff_ns": round(2 * probe["l2_atomic_ns"], 1),
        "handoff_bound_ms": round(hot["max_writes"] * 2 * probe["l2_atomic_ns"] / 1e6, 3),
        "handoff_frac": round(hot["max_writes"] * 2 * probe["l2_atomic_ns"] / 1e6 / kernel_ms, 4)}
    # L2 atomic throughput the execute kernel achieved, against distinct-word CAS
    atom_gops = stats["atomics"] / (kernel_ms / 1000.0) / 1e9
    roofline["atomics"] = {
        "achieved_gops": round(atom_gops, 4), "peak_gops": round(probe["cas_distinct_gops"], 2),
        "frac": round(atom_gops / probe["cas_distinct_gops"], 6),
        "per_batch": stats["atomics"],
        "peak_kind": "measured gcc_probe_memory cas_distinct_gops",
        "count_kind": "atomic read-modify-writes issued by the execute kernel (its own counters)"}
    sectors = {
        "bytes_per_txn": round(sect["per_txn"], 1), "achieved_gbs": round(sect_gbs, 1),
        "random_ceiling_gbs": round(probe["gather32_gbs"], 1),
        "random_gbs": round(sect["random"] / (kernel_ms / 1000.0) / 1e9, 1),
        "frac_random": round(sect["random"] / (kernel_ms / 1000.0) / 1e9 / probe["gather32_gbs"], 4),
        "ceiling_kind": "measured gcc_probe_memory gather32_gbs (random 32-byte sector reads)"}
    probe_out = {k: (round(v, 3) if isinstance(v, float) else
                     [round(x, 1) for x in v] if isinstance(v, list) else v)
                 for k, v in probe.items()}
    cpu = None
    if not args.no_cpu:
        v, info = time_oracle(table, batch, args.cpu_seconds)
        cpu = {"value": v, "unit": "txn/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole batch of {info['txns']} txns, serial in id order, "
                         f"{info['repeats']} passes, {info['seconds']} s",
               "host": host_info()}
    out = {"metric": METRIC, "value": value, "unit": "txn/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "config": config_dict(args),
           "abort_rate": stats["abort_rate"], "all_committed": committed == batch.n_txns,
           "roofline": roofline, "contention_roofline": contention, "sector_roofline": sectors,
           "memory_probe": probe_out, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock,
           "gpu_launches": launches, "schemes": schemes}
    db.close()
    return out


# ---------------------------------------------------------------------------
# batched form: 64 databases in one persistent launch
# ---------------------------------------------------------------------------
def run_batched(args, rank, world, dist=None):
    """64 key-value databases of 2^16..2^22 records (log-uniform), batches of
    1,000..262,144 txns of 4..64 ops, Zipf 0.8, OCC: one graph-replayed
    persistent launch against 64 plain launches on one stream, with launch
    parameters from the autotuner (tuned on the median batch).  Under
    torchrun every rank runs its own 64 databases (replicas): commits are
    summed over the ranks and the slowest rank's time is taken."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine as eng
    from paper_2406_10158_gb300 import workload as wl
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    t0 = time.time()
    spec = wl.batched_kv(wl.SEEDS[3] + rank, n_db=args.n_db)
    gen_s = time.time() - t0
    dbs, entries = [], []
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)).to(dev)
    for (nrec, table, batch) in spec:
        db = eng.Database("kv", n_records=nrec, n_fields=8, field_bytes=8, max_ops_per_txn=64,
                          max_batch_txns=batch.n_txns, max_batch_ops=batch.n_ops, device=dev)
        db.load_kv(table)
        e = (db, up(batch.txns), batch.n_txns, up(batch.ops), up(batch.operands), batch.n_ops,
             torch.empty(batch.n_txns * 16, dtype=torch.uint8, device=dev),
             torch.empty(batch.n_ops * 16, dtype=torch.uint8, device=dev))
        dbs.append(db)
        entries.append(e)
    torch.cuda.synchronize(dev)
    total_txns = sum(b.n_txns for (_, _, b) in spec)
    # autotune on three size classes (smallest, median, largest batch) over
    # lanes per txn {1, 2, 4, 8, 16, 32} x warps per block {1, 2, 4, 8, 16, 32}
    # x two backoff caps; the plan then takes the candidate it runs fastest
    order = sorted(range(len(spec)), key=lambda i: spec[i][2].n_txns)
    space = eng.tune_space(lanes=(1, 2, 4, 8, 16, 32), warps=(1, 2, 4, 8, 16, 32),
                           caps=(65536, 1000000), steps=2, warmup=1)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    candidates, tuned = [], []
    for cls, m in (("small", order[0]), ("median", order[len(order) // 2]), ("large", order[-1])):
        db, tx, n_t, op, od, n_o, rs, rd = entries[m]
        best_m, rep = eng.gcc_autotune(db.handle, "occ", tx.data_ptr(), n_t, op.data_ptr(),
                                       od.data_ptr(), n_o, rs.data_ptr(), rd.data_ptr(), space)
        candidates.append(best_m)
        tuned.append({"class": cls, "txns": n_t, "lanes_per_txn": best_m.lanes_per_txn,
                      "warps_per_block": best_m.warps_per_block,
                      "backoff_cap_ns": best_m.backoff_cap_ns, "report": rep})

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        return e0.elapsed_time(e1) / 1000.0

    steps = max(1, min(args.steps, 5))
    best, best_t = candidates[0], None
    for c in candidates:                              # the plan picks its own point
        pl = eng.MultiPlan("occ", entries, c)
        pl.launch(use_graph=True, stream=sh)
        t = timed(lambda: pl.launch(use_graph=True, stream=sh), 1)
        pl.close()
        if best_t is None or t < best_t:
            best, best_t = c, t

    def plain(scheme="occ", p=None):
        for (db, tx, n_t, op, od, n_o, rs, rd) in entries:
            db.execute(scheme, tx, op, od, n_t, n_o, rs, rd, p or best, sh)

    plan = eng.MultiPlan("occ", entries, best)
    plan.launch(use_graph=True, stream=sh)            # capture once
    det_plan = eng.MultiPlan("det", entries)
    det_plan.launch(use_graph=True, stream=sh)
    torch.cuda.synchronize(dev)
    with ClockSampler(dev) as clocks:
        t_plain = timed(plain, steps)
        committed_plain = sum(d.last_stats()["committed"] for d in dbs)
        t_multi = timed(lambda: plan.launch(use_graph=True, stream=sh), steps)
        committed_multi = sum(plan.stats(i)["committed"] for i in range(len(entries)))
        t_det_plain = timed(lambda: plain("det", eng.params()), steps)
        committed_det_plain = sum(d.last_stats()["committed"] for d in dbs)
        t_det = timed(lambda: det_plan.launch(use_graph=True, stream=sh), steps)
        committed_det = sum(det_plan.stats(i)["committed"] for i in range(len(entries)))
    det_plan.close()
    plan.close()
    for d in dbs:
        d.close()
    committed_plain, t_plain = replica_totals(dist, committed_plain, t_plain, dev)
    committed_multi, t_multi = replica_totals(dist, committed_multi, t_multi, dev)
    v_plain = committed_plain * steps / t_plain
    v_multi = committed_multi * steps / t_multi
    return {"metric": METRIC, "form": "batched", "value": v_multi, "unit": "txn/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000 * t_multi / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"{len(spec)} kv databases 2^16..2^22 x 8 u64, batches "
                                   f"1000..262144 txns x 4..64 ops, zipf 0.8, occ",
                       "total_txns": total_txns, "generation_s": round(gen_s, 1)},
            "plain_launches": {"value": v_plain, "unit": "txn/s",
                               "ms_per_step": 1000 * t_plain / steps},
            "speedup_vs_plain": v_multi / v_plain,
            "autotuned": {"lanes_per_txn": best.lanes_per_txn, "warps_per_block": best.warps_per_block,
                          "backoff_cap_ns": best.backoff_cap_ns, "size_classes": tuned},
            "det": {"batched_txn_per_s": committed_det * steps / t_det,
                    "plain_txn_per_s": committed_det_plain * steps / t_det_plain,
                    "speedup_vs_plain": (committed_det / t_det) / (committed_det_plain / t_det_plain),
                    "ms_per_step": 1000 * t_det / steps,
                    "all_committed": committed_det == total_txns},
            "all_committed": committed_multi == total_txns and committed_plain == total_txns,
            "clocks": clocks.summary()}


# ---------------------------------------------------------------------------
# served form: continuous batching of a Poisson trace
# ---------------------------------------------------------------------------
def sustained_rate(results):
    """The row whose latency a serving system reports: the highest offered
    rate it sustains (commits at least 98% of it), not saturation; the
    highest committed rate when none is sustained."""
    held = [r for r in results if r["committed_txn_per_s"] >= 0.98 * r["offered_txn_per_s"]]
    if held:
        return max(held, key=lambda r: r["offered_txn_per_s"])
    return max(results, key=lambda r: r["committed_txn_per_s"])


def run_served(args, rank, world):
    """Open-loop Poisson arrivals, 50/50 by count of key-value txns (2^24 x 8
    u64, 16 ops, Zipf 0.8, 80% reads) and order-entry txns (W = 8), each lane
    under its own scheme (--kv-scheme, --oe-scheme; deterministic by default),
    at each offered rate: committed txns/s and p50/p99 latency (arrival to
    result on the host), against plain per-batch launches of the same requests
    (submit, wait, next).  Each rate runs min(--requests, 10 s of arrivals)
    requests -- 10 s or 10^7 requests at the default -- taken as a prefix of
    one trace generated once.  `value` is the highest committed rate;
    `p99_latency_us` is the p99 at the highest offered rate the loop sustains
    (98% of it committed), named in `p99_at_offered_txn_per_s`."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine as eng
    from paper_2406_10158_gb300 import workload as wl
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    rates = [float(r) for r in args.rates.split(",")]
    per_rate = {r: int(min(args.requests, max(1.0, 10.0 * r))) for r in rates}
    n = max(per_rate.values())
    nrec = 1 << 24
    t_gen = time.time()
    rng = np.random.default_rng(7)
    lane_of = (rng.random(n) < 0.5).astype(np.uint32)
    n_kv, n_oe = int(np.count_nonzero(lane_of == 0)), int(np.count_nonzero(lane_of == 1))
    table = wl.kv_table_splitmix(wl.SEEDS[4], nrec, 8)
    kv = wl.kv_batch(wl.derive_seed(wl.SEEDS[4], 1), nrec=nrec, nfields=8, n_txns=max(1, n_kv),
                     read_ratio=0.8, theta=0.8)
    oe0, oe, cap = wl.order_entry(seed=wl.SEEDS[4], W=8, n_txns=max(1, n_oe))  # every rate reloads it
    trace = wl.interleave([kv, oe], lane_of)
    gen_s = time.time() - t_gen
    max_batch = args.served_max_batch
    delay_ns = args.served_delay_us * 1000
    oe_scheme = args.oe_scheme
    results = []

    def fresh():
        dkv = eng.Database("kv", n_records=nrec, n_fields=8, field_bytes=8,
                           max_batch_txns=max_batch, device=dev)
        doe = eng.Database("oe", n_warehouses=8, order_cap=cap, max_ops_per_txn=33,
                           max_batch_txns=max_batch, max_batch_ops=max_batch * 33, device=dev)
        dkv.load_kv(table)
        doe.load_oe(oe0)
        return dkv, doe

    with ClockSampler(dev) as clocks:
        for rate in rates:
            m = per_rate[rate]
            sub = trace if m == n else wl.select(trace, np.arange(m))
            arrivals = wl.poisson_arrivals(wl.SEEDS[4] + int(rate), m, rate)
            dkv, doe = fresh()
            srv = eng.Server([(dkv, args.kv_scheme, max_batch, 0, delay_ns, args.served_depth),
                              (doe, oe_scheme, max_batch, 0, delay_ns, args.served_depth)])
            comp, _ = srv.run_trace(lane_of[:m], sub, arrivals)
            tots = [srv.lane_totals(0), srv.lane_totals(1)]
            srv.close()
            dkv.close()
            doe.close()
            ok = comp["status"] == 1
            lat = (comp["done_ns"] - comp["arrival_ns"]).astype(np.float64) / 1e3
            span = (comp["done_ns"].max() - comp["arrival_ns"].min()) / 1e9
            results.append({"offered_txn_per_s": rate, "requests": m,
                            "arrival_span_s": round(float(arrivals[-1]) / 1e9, 3),
                            "committed_txn_per_s": float(ok.sum() / span),
                            "p50_latency_us": float(np.percentile(lat, 50)),
                            "p99_latency_us": float(np.percentile(lat, 99)),
                            "abort_rate": sum(t["aborts"] for t in tots) / max(1, sum(t["committed"] for t in tots)),
                            "batches": sum(t["batches"] for t in tots),
                            "all_committed": bool(ok.all())})
            del comp, sub
        # plain per-batch launches of the same requests: submit, wait, next
        dkv, doe = fresh()
        m = per_rate[max(rates)]
        lanes = lane_of[:m]
        subs = [wl.select(trace, np.nonzero(lanes == l)[0]) for l in (0, 1)]
        t0 = time.perf_counter()
        committed = 0
        for start in range(0, max(s.n_txns for s in subs), max_batch):
            for l, (db, scheme) in enumerate(((dkv, args.kv_scheme), (doe, oe_scheme))):
                idx = np.arange(start, min(start + max_batch, subs[l].n_txns))
                if idx.size:
                    _, _, st = db.run(scheme, wl.select(subs[l], idx))
                    committed += st["committed"]
        plain_s = time.perf_counter() - t0
        dkv.close()
        doe.close()
    best = max(results, key=lambda r: r["committed_txn_per_s"])
    sustained = sustained_rate(results)
    return {"metric": METRIC, "form": "served", "value": best["committed_txn_per_s"],
            "unit": "txn/s", "n_gpus": 1, "steps": len(rates), "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"50/50 kv (2^24 x 8 u64, 16 ops, zipf 0.8, 80% reads, "
                                   f"{args.kv_scheme}) and order-entry (W=8, {oe_scheme}), "
                                   f"poisson arrivals, min({args.requests}, 10 s of arrivals) "
                                   f"requests per rate",
                       "max_batch_txns": max_batch, "max_delay_us": args.served_delay_us,
                       "depth": args.served_depth,
                       "trace_generation_s": round(gen_s, 1)},
            "p99_latency_us": sustained["p99_latency_us"],
            "p99_at_offered_txn_per_s": sustained["offered_txn_per_s"], "rates": results,
            "plain_per_batch": {"value": committed / plain_s, "unit": "txn/s", "requests": m},
            "speedup_vs_plain": best["committed_txn_per_s"] / (committed / plain_s),
            "clocks": clocks.summary()}


# ---------------------------------------------------------------------------
# contention sweep: every scheme across the key-value and order-entry configs
# ---------------------------------------------------------------------------
def replay_kv_cell(db, scheme, batch, tx, op, od, rs, rd, prm) -> bool:
    """One more execution of a sweep cell's batch, replayed by the CPU oracle
    from the table it started on (the --check leg: every read value and every
    word of the final table, bit for bit)."""
    import torch
    import oracle
    from paper_2406_10158_gb300 import workload as wl
    state = db.read_kv()
    db.execute(scheme, tx, op, od, batch.n_txns, batch.n_ops, rs, rd, prm)
    torch.cuda.synchronize()
    res = rs.cpu().numpy().view(wl.RESULT_DTYPE)
    reads = rd.cpu().numpy().view(np.uint64).reshape(-1, 2)
    rep = oracle.replay_check(state, db.read_kv(), batch, res, reads, inplace=True)
    return bool(rep["ok"])


def sweep_hotspot(args, rank, eng, wl, dev, up, prm, batch_ms):
    """The sweep's hot-spot rows: uniform keys with 10% of the transactions
    writing one record, under OCC and OCC with group commit (units of 8, one
    unit per warp)."""
    import torch
    rows = []
    table, batch = wl.kv_hotspot(args.seed + rank, hot_frac=0.1)
    db = eng.Database("kv", n_records=1 << 24, n_fields=10, field_bytes=16,
                      max_batch_txns=batch.n_txns, device=dev)
    db.load_kv(table)
    tx, op, od = up(batch.txns), up(batch.ops), up(batch.operands)
    rs = torch.empty(batch.n_txns * 16, dtype=torch.uint8, device=dev)
    rd = torch.empty(batch.n_ops * 16, dtype=torch.uint8, device=dev)
    useful0 = algorithmic_bytes(batch)["bytes"]
    gc = eng.params(deadline_ns=int(args.scheme_deadline_s * 1e9), group_commit=8,
                    lanes_per_txn=32)
    for name, p_s in (("occ", prm), ("occ-group8", gc)):
        for _ in range(3):
            db.execute("occ", tx, op, od, batch.n_txns, batch.n_ops, rs, rd, p_s)
        hist = db.stage_history(2)
        st = db.last_stats()
        ms = statistics.mean(batch_ms(h) for h in hist)
        row = {"workload": "hotspot", "scheme": name,
               "committed_txn_per_s": st["committed"] / ms * 1e3,
               "abort_rate": st["abort_rate"], "ms_per_batch": ms,
               "algorithmic_gbs": useful0 / ms / 1e6,
               "all_committed": st["committed"] == batch.n_txns}
        if args.check:
            row["replayed"] = replay_kv_cell(db, "occ", batch, tx, op, od, rs, rd, p_s)
        rows.append(row)
    db.close()
    return rows


def run_sweep(args, rank, world):
    """Committed txns/s and abort rate of every scheme on the key-value
    workload (2^24 x 10 x 16-byte slots, 2^20 txns x 16 ops) at Zipf theta in
    {0, 0.6, 0.8, 0.99} x read ratio {0.5, 0.95}, of OCC with and without
    group commit on a hot spot among cold records, and of every scheme on the
    order-entry mix (2^18 txns, 50/50 NewOrder/Payment) at W in {1, 8, 64}.  Batches are
    device-resident; a batch's time is the sum of its stage events (control
    words, [deterministic preprocessing], execute, commit ranks)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_10158_gb300 import engine as eng
    from paper_2406_10158_gb300 import workload as wl
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)).to(dev)
    prm = eng.params(deadline_ns=int(args.scheme_deadline_s * 1e9))
    # the deterministic scheme three ways: per-record evaluation (prefix sums
    # for key-value, one warp per record for order entry), op by op with the
    # GPUTx waits, and op by op with every access to a record ordered (GaccO)
    variants = [(s, s, prm) for s in SCHEMES] + [
        ("det-dataflow", "det", eng.params(deadline_ns=int(args.scheme_deadline_s * 1e9),
                                           det_dataflow=1)),
        ("det-gacco", "det", eng.params(deadline_ns=int(args.scheme_deadline_s * 1e9),
                                        det_dataflow=2))]

    def batch_ms(h):
        return h["prep_ms"] + h["kernel_ms"] + h["order_ms"]

    kv_rows, oe_rows, hot_rows = [], [], []
    parts = set(args.sweep_parts.split(","))
    with ClockSampler(dev) as clocks:
        for rr in ((0.5, 0.95) if "kv" in parts else ()):
            for theta in (0.0, 0.6, 0.8, 0.99):
                table, batch = wl.ycsb_kv(args.seed + rank, theta=theta, read_ratio=rr)
                db = eng.Database("kv", n_records=1 << 24, n_fields=10, field_bytes=16,
                                  max_batch_txns=batch.n_txns, device=dev)
                db.load_kv(table)
                tx, op, od = up(batch.txns), up(batch.ops), up(batch.operands)
                rs = torch.empty(batch.n_txns * 16, dtype=torch.uint8, device=dev)
                rd = torch.empty(batch.n_ops * 16, dtype=torch.uint8, device=dev)
                torch.cuda.synchronize(dev)
                useful0 = algorithmic_bytes(batch)["bytes"]
                useful_mv = mvcc_algorithmic_bytes(batch)["bytes"]
                reps = 1 if theta >= 0.99 else 3
                for name, scheme, p_s in variants:
                    for _ in range(1 + reps):
                        db.execute(scheme, tx, op, od, batch.n_txns, batch.n_ops, rs, rd, p_s)
                    hist = db.stage_history(reps)
                    st = db.last_stats()
                    ms = statistics.mean(batch_ms(h) for h in hist)
                    useful = useful_mv if scheme == "mvcc" else useful0
                    row = {"theta": theta, "read_ratio": rr, "scheme": name,
                           "committed_txn_per_s": st["committed"] / ms * 1e3,
                           "abort_rate": st["abort_rate"], "ms_per_batch": ms,
                           "algorithmic_gbs": useful / ms / 1e6,
                           "all_committed": st["committed"] == batch.n_txns}
                    if args.check:
                        row["replayed"] = replay_kv_cell(db, scheme, batch, tx, op, od, rs, rd,
                                                         p_s)
                    kv_rows.append(row)
                db.close()
        # one hot spot among cold records: OCC against OCC with group commit
        for _ in range(1 if "hotspot" in parts else 0):
            hot_rows += sweep_hotspot(args, rank, eng, wl, dev, up, prm, batch_ms)
        for W in ((1, 8, 64) if "oe" in parts else ()):
            db0, batch, cap = wl.order_entry(W=W, n_txns=1 << 18)
            db = eng.Database("oe", n_warehouses=W, order_cap=cap, max_ops_per_txn=33,
                              max_batch_txns=batch.n_txns, max_batch_ops=batch.n_ops, device=dev)
            tx, op, od = up(batch.txns), up(batch.ops), up(batch.operands)
            rs = torch.empty(batch.n_txns * 16, dtype=torch.uint8, device=dev)
            rd = torch.empty(batch.n_ops * 16, dtype=torch.uint8, device=dev)
            useful = oe_algorithmic_bytes(batch)["bytes"]
            for name, scheme, p_s in variants:
                if scheme == "mvcc":
                    continue                       # key-value only
                for _ in range(2):                 # a warm-up batch, then the timed one
                    db.load_oe(db0)               # fresh order slots for the inserts
                    torch.cuda.synchronize(dev)
                    db.execute(scheme, tx, op, od, batch.n_txns, batch.n_ops, rs, rd, p_s)
                h = db.stage_history(1)[-1]
                st = db.last_stats()
                ms = batch_ms(h)
                row = {"W": W, "scheme": name,
                       "committed_txn_per_s": st["committed"] / ms * 1e3,
                       "abort_rate": st["abort_rate"], "ms_per_batch": ms,
                       "algorithmic_gbs": useful / ms / 1e6,
                       "all_committed": st["committed"] == batch.n_txns}
                if args.check:
                    import oracle
                    torch.cuda.synchronize(dev)
                    res = rs.cpu().numpy().view(wl.RESULT_DTYPE)
                    reads = rd.cpu().numpy().view(np.uint64).reshape(-1, 2)
                    rep = oracle.oe_replay_check(db0, db.read_oe(), W, cap, batch, res, reads)
                    row["replayed"] = bool(rep["ok"]) and oracle.oe_consistency(
                        db.read_oe(), W, cap) == 0
                oe_rows.append(row)
            db.close()
    head = next((r for r in kv_rows if r["theta"] == 0.8 and r["read_ratio"] == 0.5
                 and r["scheme"] == "occ"), None)
    return {"metric": METRIC, "form": "sweep",
            "value": head["committed_txn_per_s"] if head else None,
            "unit": "txn/s", "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "kv 2^24 x 10 x 16 B, 2^20 txns x 16 ops, zipf {0,0.6,0.8,0.99}"
                                   " x read ratio {0.5,0.95}; the same with uniform keys and 10%"
                                   " of the txns writing one record (hotspot: occ, occ with"
                                   " group commit); order-entry W {1,8,64}, 2^18 txns",
                       "value_is": "occ at zipf 0.8, read ratio 0.5"},
            "kv": kv_rows, "hotspot": hot_rows, "order_entry": oe_rows,
            "clocks": clocks.summary()}


def main(argv=None):
    args = parse_args(argv)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference" and rank != 0:
        return                       # the CPU oracle runs on rank 0 only
    one_gpu_form = args.form in ("served", "sweep")
    if args.impl == "ours" and one_gpu_form and rank != 0:
        return                       # the served form and the sweep run on one GPU
    if world > 1 and args.impl == "ours" and not one_gpu_form:
        # replicas: the process group only carries the timing barrier and max
        import torch
        import torch.distributed as dist_mod
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.form == "batched":
        out = run_batched(args, rank, world, dist)
    elif args.form == "served":
        out = run_served(args, rank, world)
    elif args.form == "sweep":
        out = run_sweep(args, rank, world)
    else:
        out = run_ours(args, rank, world, dist)
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
