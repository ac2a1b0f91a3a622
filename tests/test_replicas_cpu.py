"""The bench's N-GPU mode on the CPU: two gloo ranks run the replica
bookkeeping of bench.py (barrier, slowest rank's time, sum of the ranks'
certified solves), and the reference arm leaves every rank but 0 idle.

The path does not shard (every rank solves its own copy of the workload), so
these are the only multi-rank parts; they need no GPU."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, units, seconds):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        r = bench.Replicas(dist, world, "cpu")
        r.barrier()
        assert r.max(seconds[rank]) == max(seconds)
        assert r.sum(units[rank]) == sum(units)
        # whole-job throughput: all ranks' units over the slowest rank's time
        assert r.throughput(units[rank], seconds[rank]) == pytest.approx(sum(units) / max(seconds), rel=1e-15)
        r.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("units,seconds", [((200.0, 200.0), (0.08, 0.11)), ((195.0, 200.0), (0.30, 0.25))])
def test_two_gloo_ranks_combine_time_and_units(units, seconds):
    mp.spawn(_rank_main, args=(2, _free_port(), units, seconds), nprocs=2, join=True)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Replicas()
    r.barrier()
    assert r.max(0.5) == 0.5 and r.sum(3.0) == 3.0 and r.throughput(200.0, 0.1) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank but 0 exits without work or output."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(bench.parse())
    assert out.getvalue() == ""
