"""The multi-GPU path is replicas only: every rank runs its own database and
batch, and the process group carries the timing barrier and the totals.
These tests run that host logic as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r committed 100 * (r + 1) transactions in 10 * (r + 1) ms
        c, t = bench.replica_totals(dist, 100.0 * (rank + 1), 10.0 * (rank + 1))
        out[rank] = (c, t)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_totals_sum_commits_and_take_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    # every rank sees the job totals: 100 + 200 commits, the slower rank's 20 ms
    assert dict(out) == {0: (300.0, 20.0), 1: (300.0, 20.0)}


def test_replica_totals_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(None, 123.0, 4.5) == (123.0, 4.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle (the reference arm) runs on rank 0 alone; the
    other ranks return at once without output."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference"]) is None
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("form", ["served", "sweep"])
def test_one_gpu_forms_run_on_rank_zero_only(monkeypatch, capsys, form):
    """The served form and the sweep are single-GPU measurements: under
    torchrun the other ranks return at once, and no process group is made."""
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    calls = []
    monkeypatch.setattr(bench, "run_served", lambda *a: calls.append("served") or None)
    monkeypatch.setattr(bench, "run_sweep", lambda *a: calls.append("sweep") or None)
    monkeypatch.setattr(dist, "init_process_group",
                        lambda *a, **k: pytest.fail("no process group for a one-GPU form"))
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.main(["--form", form]) is None
    assert calls == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.main(["--form", form])
    assert calls == [form]


def test_batched_form_gets_the_process_group(monkeypatch):
    """The batched form runs on every rank and receives the process group for
    its barriers and totals."""
    sys.path.insert(0, ROOT)
    import bench
    seen = []
    monkeypatch.setattr(bench, "run_batched", lambda args, rank, world, dist: seen.append(
        (rank, world, dist)) or None)
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    bench.main(["--form", "batched"])
    assert seen == [(0, 1, None)]
