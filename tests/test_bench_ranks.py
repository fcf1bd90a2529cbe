"""The multi-rank logic of bench.py on CPU: two ranks over gloo (127.0.0.1).

bench.py runs one planner per GPU (weak scaling): every rank plans its own problem, the
slowest rank's time is the job's time, throughputs add up, and the reference arm runs
on rank 0 only.  These paths are exercised here with gloo instead of NCCL; no GPU is used.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        res = {
            "max": b.max_over_ranks([1.0 + rank, 5.0 - rank, 0.25 * rank], world, "cpu"),
            "sum": b.sum_over_ranks([100.0 * (rank + 1)], world, "cpu"),
            "session": b.rank_session(rank),
            "session_7": b.rank_session(rank, 7),
        }
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_ranks_take_the_slowest_time_and_add_throughput(tmp_path):
    torch_mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    torch_mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    assert r[0]["max"] == r[1]["max"] == [2.0, 5.0, 0.25]
    assert r[0]["sum"] == r[1]["sum"] == [300.0]
    # independent problems: distinct Philox session words per rank, and per session within a rank
    assert r[0]["session"] != r[1]["session"]
    assert len({r[0]["session_7"], r[1]["session_7"], r[0]["session"], r[1]["session"]}) == 4


def test_weak_scaling_value_counts_every_rank():
    assert bench.weak_value(13_107_200, 2, 0.5) == pytest.approx(2 * 13_107_200 / 0.5)
    assert bench.weak_value(10.0, 1, 2.0) == 5.0
    assert bench.max_over_ranks([1.5, 2], 1, "cpu") == [1.5, 2.0]


def test_reference_arm_runs_on_rank_zero_only():
    class A:
        workload = "roofline"
        steps = 1
        warmup = 0
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(A(), 2, 1, 1) is None
    assert buf.getvalue() == ""
